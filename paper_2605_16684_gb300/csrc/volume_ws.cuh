// volume_ws.cuh -- the warp-specialised mixed-precision volume kernel (single
// meshes with a hydrostatic background).
//
// In the mixed path a tile's node work (the prologue, FP64 differences
// against the background, and the epilogue, the FP64 state update) runs on
// the FP64 pipe, which this GPU issues at 2 lanes per cycle per SM, while the
// pair pass runs on the FP32 pipe.  With one set of warps walking the phases
// in turn, each pipe idles while the other works.  Here the CTA holds two
// roles.  Consumer warps (one thread per pencil) run the pair pass of tile k
// and then the FP32 part of its stage update (-1/J times the sums, the
// background's right-hand side, the Coriolis source, the new FP32 increment
// dq).  Producer warps run the prologue of tile k + 1 and the FP64 part of
// tile k - 1's update (q += B dq and the stores).  One copy warp issues the
// bulk copies (a copy issue can stall its warp for a thousand cycles while
// the copy engine is busy; here that stalls no compute).
// The node fields S and the FP64 state copy are double buffered; each buffer
// is handed over with an mbarrier (sfull: producers -> consumers, node fields
// ready; rfull: consumers -> producers, increments ready).  Every wait is
// bounded: on a timeout the role agrees on it with a role-wide barrier
// reduction, sets the kernel's timeout flag and leaves; the other role's
// bounded waits then run out too.  The arithmetic is that of volume_pairs.cuh
// in the same order, so results are bitwise those of k_volume_pipe32.
#pragma once
#include "volume_pipe.cuh"

namespace esdg_vol {

// named barriers (id 0 is __syncthreads) and role-wide decisions
__device__ __forceinline__ void ws_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool ws_bar_or(bool pred, int id, int n) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, %2, %3, a;\n"
      " selp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
// plain arrival (release at CTA scope) on a count-1 mbarrier
__device__ __forceinline__ void ws_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(esdg_smem_addr(bar)) : "memory");
}

// copy issue by the copy warp: lanes [FIRST, FIRST + 32)
template <int FIRST_>
struct WsIssuers {
  static constexpr int FIRST = FIRST_, COUNT = 32;
  static __device__ __forceinline__ unsigned mask() { return 0xffffffffu; }
  static __device__ __forceinline__ bool is(int tid) { return tid >= FIRST && tid < FIRST + 32; }
};

// Tile shape (elements per tile) and producer warps per order; consumers are
// the pencil threads of the tile rounded up to whole warps.
template <int N>
struct WsCfg {
  static constexpr bool ON = false;
  static constexpr int EPB = 1, PW = 1;
};
#ifndef ESDG_WS4_EPB
#define ESDG_WS4_EPB 4
#endif
#ifndef ESDG_WS4_PW
#define ESDG_WS4_PW 5
#endif
template <>
struct WsCfg<4> {
  static constexpr bool ON = true;
  // 300 pencils in 10 warps, 5 producer warps, 1 copy warp
  static constexpr int EPB = ESDG_WS4_EPB, PW = ESDG_WS4_PW;
};

template <int N, int MODE>
struct Ws32 {
  using SH = Shape<N, true, true, WsCfg<N>::EPB>;
  static constexpr int NP = SH::NP, EPB = SH::EPB, P = NP * EPB, NF = SH::NF;
  static constexpr int CT = SH::THREADS;          // consumer threads
  static constexpr int PT = 32 * WsCfg<N>::PW;    // producer threads
  static constexpr int T = CT + PT + 32;          // and the copy warp
  static constexpr int up16(int b) { return (b + 15) & ~15; }
  // byte offsets, 16-byte aligned; bulk-copy targets hold 32 extra bytes
  static constexpr int RAW_Q = 0;                                    // [el][5][NP]  double
  static constexpr int RAW_BG = up16(RAW_Q + 8 * (5 * P + 4));       // [el][3][NP]  double
  static constexpr int RAW_BGP = up16(RAW_BG + 8 * (3 * P + 4));     // [el][4][NP]  float
  static constexpr int RAW_G = up16(RAW_BGP + 4 * (4 * P + 8));      // [el][11][NP] float
  static constexpr int SB = up16(4 * NF * P);                        // one node-field buffer
  static constexpr int S0 = up16(RAW_G + 4 * (ESDG_NVGEO * P + 8));  // 2 x [el][NF][NP] float
  static constexpr int QB = 8 * 5 * P;                               // one state-copy buffer
  static constexpr int EPQ = S0 + 2 * SB;                            // 2 x [el][5][NP] double
  static constexpr int JB = up16(4 * P);
  static constexpr int EPJ = EPQ + 2 * QB;                           // 2 x [el][NP] float
  static constexpr int CUR_RB = up16(EPJ + 2 * JB);                  // [el][3][NP]  float
  static constexpr int CUR_DQ = up16(CUR_RB + 4 * (3 * P + 8));      // [el][5][NP]  float
  static constexpr int TOTAL = MODE ? up16(CUR_DQ + 4 * (5 * P + 8)) : CUR_DQ;
  static constexpr size_t SMEM = (size_t)TOTAL;
  // after the pair pass, node fields 15.. of a buffer are free: the stage
  // increment (or the FP32 right-hand side) of each node goes there
  static constexpr int F_INC = 15;
  static_assert(F_INC + 5 <= NF, "room for the increment");
};

template <int EPB>
struct WsCtl {
  unsigned long long raw, cur;        // bulk copies: next tile's data, current tile's dq / rhs_bg
  unsigned long long rawfree;         // the tile's data consumed (producers -> copy warp)
  unsigned long long sfull[2];        // node fields of a buffer ready (producers -> consumers)
  unsigned long long rfull[2];        // increments of a buffer ready (consumers -> producers)
  int4 info[2];                       // tile of a buffer: (0, first element, elements)
  int logs[2];                        // the buffer's tile needs the logarithm branch
  float phi0[2][EPB];                 // each element's reference geopotential
  EsdgMember desc;
};

template <int N, int MODE>
__global__ void __launch_bounds__(Ws32<N, MODE>::T, 1)
    k_volume_ws32(const EsdgMember one, int ntiles, EsdgLGL L, double rkA, double rkB,
                  unsigned phantom, int t1, int s1) {
  using W = Ws32<N, MODE>;
  using SH = typename W::SH;
  constexpr int Nq = SH::Nq, NP = SH::NP, NPEN = SH::NPEN, EPB = SH::EPB, NF = SH::NF;
  constexpr int CT = W::CT, PT = W::PT, NN = EPB * NP, FI = W::F_INC;
  constexpr int PBAR = 1, CBAR = 2;  // named barriers of the producer and consumer roles
  using ISS = WsIssuers<CT + PT>;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) WsCtl<EPB> c;
  double* const rawq = reinterpret_cast<double*>(smraw + W::RAW_Q);
  double* const rawbg = reinterpret_cast<double*>(smraw + W::RAW_BG);
  float* const rawbgp = reinterpret_cast<float*>(smraw + W::RAW_BGP);
  float* const rawg = reinterpret_cast<float*>(smraw + W::RAW_G);
  float* const currb = reinterpret_cast<float*>(smraw + W::CUR_RB);
  float* const curdq = reinterpret_cast<float*>(smraw + W::CUR_DQ);
  auto Sbuf = [&](int b) { return reinterpret_cast<float*>(smraw + W::S0 + b * W::SB); };
  auto Qbuf = [&](int b) { return reinterpret_cast<double*>(smraw + W::EPQ + b * W::QB); };
  auto Jbuf = [&](int b) { return reinterpret_cast<float*>(smraw + W::EPJ + b * W::JB); };
  const int tid = threadIdx.x;
  if (tid == 0) {
    // copy barriers: the expect_tx arrival + the copy warp's cp.async arrivals
    esdg_mbar_init(&c.raw, 1 + ISS::COUNT);
    esdg_mbar_init(&c.cur, 1 + ISS::COUNT);
    esdg_mbar_init(&c.rawfree, 1);
    for (int b = 0; b < 2; b++) {
      esdg_mbar_init(&c.sfull[b], 1);
      esdg_mbar_init(&c.rfull[b], 1);
    }
    esdg_fence_mbar_init();
    c.desc = one;
  }
  __syncthreads();
  const EsdgGrid& g = c.desc.g;
  const EsdgVolArgs& a = c.desc.a;
  // this CTA's tiles: blockIdx.x + k gridDim.x, k = 0 .. K - 1
  const int K = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto tile_of = [&](int k) {
    return pipe_tile<false, EPB>(nullptr, (int)blockIdx.x + k * (int)gridDim.x, t1, s1, g.E);
  };
  const double* const q_in = a.q_in;
  const double* const bgd = a.bg;
  const float* const bgp = a.bgp;
  const float* const vg = reinterpret_cast<const float*>(a.vgeo);

  if (tid >= CT + PT) {
    // ===================== the copy warp =====================================
    auto issue_raw = [&](int k, unsigned ph) {
      const int4 tr = tile_of(k);
      const int e0 = tr.y, ne = tr.z, E = g.E;
      const BlockCopy bl[4] = {
          {rawq, q_in + (size_t)e0 * 5 * NP, q_in + (size_t)E * 5 * NP, ne * 5 * NP, 8},
          {rawbg, bgd + (size_t)e0 * 3 * NP, bgd + (size_t)E * 3 * NP, ne * 3 * NP, 8},
          {rawbgp, bgp + (size_t)e0 * 4 * NP, bgp + (size_t)E * 4 * NP, ne * 4 * NP, 4},
          {rawg, vg + (size_t)e0 * ESDG_NVGEO * NP, vg + (size_t)E * ESDG_NVGEO * NP,
           ne * ESDG_NVGEO * NP, 4}};
      pipe_issue<ISS>(tid, bl, 4, &c.raw, 0, nullptr, nullptr, ph, true);
    };
    // the tile's background rhs and dq, read by the consumers
    auto issue_cur = [&](int k) {
      const int4 tr = tile_of(k);
      const int e0 = tr.y, ne = tr.z, E = g.E;
      const float* dqg = reinterpret_cast<const float*>(a.dq);
      const BlockCopy cb[2] = {
          {currb, a.rhs_bg + (size_t)e0 * 3 * NP, a.rhs_bg + (size_t)E * 3 * NP, ne * 3 * NP, 4},
          {curdq, dqg + (size_t)e0 * 5 * NP, dqg + (size_t)E * 5 * NP, MODE ? ne * 5 * NP : 0, 4}};
      pipe_issue<ISS>(tid, cb, 2, &c.cur, 0, nullptr, nullptr, 0, true);
    };
    int nr = 0, nc = 0;  // copies issued (RAW, CUR)
    if (K > 0) {
      issue_raw(0, phantom);
      issue_cur(0);
      nr = nc = 1;
    }
    // RAW(k) consumed -> RAW(k + 1); CUR(k) consumed (the tile's increments are
    // ready) -> CUR(k + 1).  Every copy issued is waited for by another role
    // before the signal that frees its buffer, except on a timeout.
    bool ok = true;
    for (int k = 0; k + 1 < K; k++) {
      ok = esdg_mbar_wait(&c.rawfree, k & 1, ESDG_WAIT_LIMIT);
      if (!ok) break;
      issue_raw(k + 1, 0);
      nr++;
      ok = esdg_mbar_wait(&c.rfull[k & 1], (k >> 1) & 1, ESDG_WAIT_LIMIT);
      if (!ok) break;
      issue_cur(k + 1);
      nc++;
    }
    esdg_cp_async_wait_all();
    if (!ok) {
      // a role stopped: the last copies issued may still be landing in this
      // CTA's shared memory; wait for them (bounded; a phase that completed
      // already returns at once) before leaving
      if ((tid & 31) == 0) atomicExch(&g_esdg_vol_timeout, 1);
      esdg_mbar_wait(&c.raw, (nr - 1) & 1, ESDG_WAIT_LIMIT);
      esdg_mbar_wait(&c.cur, (nc - 1) & 1, ESDG_WAIT_LIMIT);
    }
  } else if (tid >= CT) {
    // ===================== producers: prologue, FP64 update ==================
    const int p = tid - CT;
    const EsdgPhys Pl = c.desc.P;
    const float gm1f = esdg_d2f(Pl.gamma - 1.0);
    for (int k = 0; k <= K; k++) {
      if (k < K) {
        // ---- prologue of tile k into buffer k & 1 ----------------------------
        const int b = k & 1;
        const bool ok = esdg_mbar_wait(&c.raw, k & 1, ESDG_WAIT_LIMIT);
        if (ws_bar_or(!ok, PBAR, PT)) {
          if (p == 0) atomicExch(&g_esdg_vol_timeout, 1);
          break;
        }
        const int4 tr = tile_of(k);
        const int e0 = tr.y, ne = tr.z;
        float* const sm = Sbuf(b);
        double* const epq = Qbuf(b);
        float* const epj = Jbuf(b);
        const double* qr0 = rawq + esdg_block_shift(q_in + (size_t)e0 * 5 * NP);
        const double* br0 = rawbg + esdg_block_shift(bgd + (size_t)e0 * 3 * NP);
        const float* pr0 = rawbgp + esdg_block_shift(bgp + (size_t)e0 * 4 * NP);
        const float* gr0 = rawg + esdg_block_shift(vg + (size_t)e0 * ESDG_NVGEO * NP);
        struct In {
          double q0, q1, q2, q3, q4, rb, eb, phi;
          float b0, b1, b2, b3, phh;
          int el, n;
          bool live, any;
        };
        auto load = [&](int idx) {
          In x;
          x.any = idx < NN;
          x.el = idx / NP;
          x.n = idx - x.el * NP;
          x.live = x.any && x.el < ne;
          const int el = x.live ? x.el : 0, n = x.live ? x.n : 0;
          const double* qr = qr0 + (size_t)el * 5 * NP + n;
          const double* br = br0 + (size_t)el * 3 * NP + n;
          const float* pr = pr0 + (size_t)el * 4 * NP + n;
          x.q0 = qr[0];
          x.q1 = qr[NP];
          x.q2 = qr[2 * NP];
          x.q3 = qr[3 * NP];
          x.q4 = qr[4 * NP];
          x.rb = br[0];
          x.eb = br[NP];
          x.phi = br[2 * NP];
          x.b0 = pr[0];
          x.b1 = pr[NP];
          x.b2 = pr[2 * NP];
          x.b3 = pr[3 * NP];
          x.phh = gr0[((size_t)el * ESDG_NVGEO + 10) * NP + n];
          return x;
        };
        auto store = [&](const In& x, const Prim32& o) {
          if (!x.any) return;
          const int el = x.el, n = x.n;
          float* S = sm + (size_t)el * NF * NP;
          if (x.live) {
#pragma unroll
            for (int f = 0; f < 7; f++) {
              S[f * NP + n] = o.s[f];
              S[(SH::F_BG + f) * NP + n] = o.bgf[f];
            }
            const float* gr = gr0 + (size_t)el * ESDG_NVGEO * NP + n;
#pragma unroll
            for (int f = 0; f < 9; f++) S[(SH::F_NH + f) * NP + n] = gr[f * NP];
            double* X = epq + (size_t)el * 5 * NP + n;
            X[0] = x.q0;
            X[NP] = x.q1;
            X[2 * NP] = x.q2;
            X[3 * NP] = x.q3;
            X[4 * NP] = x.q4;
            epj[(size_t)el * NP + n] = gr[9 * NP];
            if (n == 0) c.phi0[b][el] = esdg_d2f(x.phi);
          } else {  // padding element: any valid state, results are discarded
            S[0 * NP + n] = 0.25f;
            S[1 * NP + n] = 0.5f;
            S[2 * NP + n] = 1.0f;
            for (int f = 3; f < NF; f++) S[f * NP + n] = 0.0f;
          }
        };
        auto prim = [&](const In& x) {
          return prims32bg(x.q0, x.q1, x.q2, x.q3, x.q4, x.phi, x.phh, gm1f, x.rb, x.eb, x.b0,
                           x.b1, x.b2, x.b3);
        };
        // two nodes per thread and round; a warp whose second slots all lie
        // past the tile (warp-uniform test on its first lane) converts one
        for (int i0 = p; i0 < NN; i0 += 2 * PT) {
          if (i0 - (p & 31) + PT < NN) {
            const In x0 = load(i0), x1 = load(i0 + PT);
            const Prim32 o0 = prim(x0), o1 = prim(x1);
            store(x0, o0);
            store(x1, o1);
          } else {
            const In x0 = load(i0);
            store(x0, prim(x0));
          }
        }
        ws_bar(PBAR, PT);  // node fields written; RAW consumed
        if (p == 0) ws_arrive(&c.rawfree);
        int need = 0;
        for (int idx = p; idx < NN; idx += PT) {
          const int el2 = idx / NP, n = idx - el2 * NP;
          const float* S = sm + (size_t)el2 * NF * NP;
          const float r0 = S[0], rn = S[n], b0 = S[NP], bn = S[NP + n];
          // |f| < 0.14 keeps u < ESDG_LOG_EPS32 for every pair
          if (fabsf(rn - r0) > 0.13f * r0 || fabsf(bn - b0) > 0.13f * b0) need = 1;
        }
        need = ws_bar_or(need, PBAR, PT);
        if (p == 0) {
          c.info[b] = tr;
          c.logs[b] = need;
          ws_arrive(&c.sfull[b]);
        }
      }
      if (k >= 1) {
        // ---- FP64 update of tile k - 1 from buffer (k - 1) & 1 ------------------
        const int kk = k - 1, b = kk & 1;
        const bool okr = esdg_mbar_wait(&c.rfull[b], (kk >> 1) & 1, ESDG_WAIT_LIMIT);
        if (ws_bar_or(!okr, PBAR, PT)) {
          if (p == 0) atomicExch(&g_esdg_vol_timeout, 1);
          break;
        }
        const int4 tr = tile_of(kk);
        const int e0 = tr.y, ne = tr.z;
        const float* const sm = Sbuf(b);
        const double* const epq = Qbuf(b);
        const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
        const double* xg = a.x;
        float* const dqp = reinterpret_cast<float*>(a.dq);
        double* const qio = a.q_io;
        double* const rhsp = a.rhs;
        int* const status = a.status;
        const float Bf = esdg_d2f(rkB);
        bool bad = false;
        // all of a thread's nodes at once: loads, then arithmetic, then stores
        constexpr int R = (NN + PT - 1) / PT;
        float dv[R][5];
        double xq[R][5];
#pragma unroll
        for (int h = 0; h < R; h++) {
          const int idx = p + h * PT;
          const int el2 = idx / NP, n = idx - el2 * NP;
          const bool live = idx < NN && el2 < ne;
          const float* S = sm + (size_t)(live ? el2 : 0) * NF * NP + FI * NP + (live ? n : 0);
          const double* X = epq + (size_t)(live ? el2 : 0) * 5 * NP + (live ? n : 0);
#pragma unroll
          for (int v = 0; v < 5; v++) {
            dv[h][v] = S[v * NP];
            xq[h][v] = X[v * NP];
          }
        }
#pragma unroll
        for (int h = 0; h < R; h++) {
          const int idx = p + h * PT;
          const int el2 = idx / NP, n = idx - el2 * NP, e2 = e0 + el2;
          if (idx >= NN || el2 >= ne) continue;
          const size_t qb = (size_t)e2 * 5 * NP + n;
          if constexpr (MODE != 0) {
#pragma unroll
            for (int v = 0; v < 5; v++) {
              dqp[qb + (size_t)v * NP] = dv[h][v];
              const double qn = xq[h][v] + esdg_f2d(Bf * dv[h][v]);
              qio[qb + (size_t)v * NP] = qn;
              bad |= esdg_bad_state(qn, v == 0);
            }
          } else {  // right-hand side in FP64
            double r[5];
#pragma unroll
            for (int v = 0; v < 5; v++) r[v] = esdg_f2d(dv[h][v]);
            if (rot) {
              const double y = xg[((size_t)e2 * 3 + 1) * NP + n];
              const double f = Pl.f0 + Pl.beta * (y - Pl.y0);
              r[1] = fma(f, xq[h][2], r[1]);
              r[2] = fma(-f, xq[h][1], r[2]);
            }
#pragma unroll
            for (int v = 0; v < 5; v++) rhsp[qb + (size_t)v * NP] = r[v];
          }
        }
        if (MODE != 0 && bad && status) *status = 1;
        ws_bar(PBAR, PT);  // the buffer's increments read
      }
    }
  } else {
    // ===================== consumers: pair pass and FP32 stage part ==========
    const bool active = tid < SH::PENCILS;
    const int el = active ? tid / (3 * NPEN) : 0;
    const int rr = tid - el * 3 * NPEN;
    const int d = active ? rr / NPEN : 0;
    const int pen = rr - d * NPEN;
    const int ps = pen % Nq, pt = pen / Nq;
    const int stride = (d == 0) ? 1 : ((d == 1) ? Nq : Nq * Nq);
    const int base = (d == 0) ? Nq * (ps + Nq * pt) : ((d == 1) ? (ps + Nq * Nq * pt) : (ps + Nq * pt));
    const EsdgPhys Pl = c.desc.P;
    const float ce = esdg_d2f(0.5 * Pl.igm1);
    const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
    const float Af = esdg_d2f(rkA), dtf = esdg_d2f(a.dt);
    for (int k = 0; k < K; k++) {
      const int b = k & 1;
      const bool ok = esdg_mbar_wait(&c.sfull[b], (k >> 1) & 1, ESDG_WAIT_LIMIT);
      if (ws_bar_or(!ok, CBAR, CT)) {
        if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
        break;
      }
      const int e0 = c.info[b].y, ne = c.info[b].z;
      const int need_logs = c.logs[b];
      float* const Sb = Sbuf(b);
      float acc[Nq][5];
#pragma unroll
      for (int i = 0; i < Nq; i++)
#pragma unroll
        for (int v = 0; v < 5; v++) acc[i][v] = 0.0f;
      if (active && el < ne) {
        const FaceTerms<float> ft = face_fetch<N, float>(g, a, e0 + el, d, ps + Nq * pt);
        const float* S = Sb + (size_t)el * NF * NP;
        if (need_logs)
          pencil_pass<N, true, true, true>(S, d, base, stride, L, ce, acc);
        else
          pencil_pass<N, true, false, true>(S, d, base, stride, L, ce, acc);
        const float phi0 = c.phi0[b][el];
#pragma unroll
        for (int i = 0; i < Nq; i++) acc[i][4] = fmaf(phi0, acc[i][0], acc[i][4]);
        face_add<N, float>(ft, acc);
      }
      ws_bar(CBAR, CT);  // every node field of the buffer read
      if (active && el < ne) {
        float* S = Sb + (size_t)el * NF * NP;
#pragma unroll
        for (int i = 0; i < Nq; i++)
#pragma unroll
          for (int v = 0; v < 5; v++) S[(d * 5 + v) * NP + base + i * stride] = acc[i][v];
      }
      // the tile's background rhs and dq
      const bool okc = esdg_mbar_wait(&c.cur, k & 1, ESDG_WAIT_LIMIT);
      if (ws_bar_or(!okc, CBAR, CT)) {  // also: every sum written
        if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
        break;
      }
      // FP32 part of the stage update (stage32's order), node by node
      const float* RB0 = currb + esdg_block_shift(a.rhs_bg + (size_t)e0 * 3 * NP);
      const float* D0 =
          curdq + esdg_block_shift(reinterpret_cast<const float*>(a.dq) + (size_t)e0 * 5 * NP);
      const float* const epj = Jbuf(b);
      const double* const epq = Qbuf(b);
      for (int idx = tid; idx < NN; idx += CT) {
        const int el2 = idx / NP, n = idx - el2 * NP;
        if (el2 >= ne) continue;
        float* S = Sb + (size_t)el2 * NF * NP;
        const float iJ = epj[(size_t)el2 * NP + n];
        const float* RB = RB0 + (size_t)el2 * 3 * NP + n;
        float r[5];
#pragma unroll
        for (int v = 0; v < 5; v++)
          r[v] = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
        if constexpr (MODE != 0) {
          r[1] += RB[0];
          r[2] += RB[NP];
          r[3] += RB[2 * NP];
          if (rot) {
            const double y = a.x[((size_t)(e0 + el2) * 3 + 1) * NP + n];
            const float f = esdg_d2f(Pl.f0 + Pl.beta * (y - Pl.y0));
            const double* X = epq + (size_t)el2 * 5 * NP + n;
            r[1] = fmaf(f, esdg_d2f(X[2 * NP]), r[1]);
            r[2] = fmaf(-f, esdg_d2f(X[NP]), r[2]);
          }
          const float* Dq = D0 + (size_t)el2 * 5 * NP + n;
#pragma unroll
          for (int v = 0; v < 5; v++) {
            // first stage (A = 0): the register is not read (see stage32)
            const float dv = Af == 0.0f ? dtf * r[v] : fmaf(Af, Dq[v * NP], dtf * r[v]);
            S[(FI + v) * NP + n] = dv;
          }
        } else {
#pragma unroll
          for (int v = 0; v < 5; v++)
            S[(FI + v) * NP + n] = r[v] + (v >= 1 && v <= 3 ? RB[(v - 1) * NP] : 0.0f);
        }
      }
      ws_bar(CBAR, CT);  // increments written, CUR read
      if (tid == 0) ws_arrive(&c.rfull[b]);
    }
  }
}

template <int N, int MODE>
cudaError_t launch_ws32(const EsdgGrid& g, const EsdgPhys& P, const EsdgLGL& L,
                        const EsdgVolArgs& a, cudaStream_t s) {
  using W = Ws32<N, MODE>;
  constexpr auto k = k_volume_ws32<N, MODE>;
  const int cap = pipe_grid_cap<k>(W::T, W::SMEM);
  if (cap < 0) return cudaErrorInvalidConfiguration;
  int ntiles, grid, t1, s1;
  pipe_split(g.E, W::EPB, cap, ntiles, grid, t1, s1);
  if (ntiles == 0) return cudaSuccess;
  k<<<grid, W::T, W::SMEM, s>>>(pipe_member(g, P, a), ntiles, L, a.rkA, a.rkB, esdg_take_phantom(),
                                t1, s1);
  return cudaGetLastError();
}

}  // namespace esdg_vol
