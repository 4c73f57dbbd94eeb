// volume_pipe.cuh -- the pipelined persistent volume kernels (FP64 and mixed):
// one CTA per SM walks its tiles while the copy engine prefetches the next
// tile; single meshes or batch work tables; their launchers.
#pragma once
#include "volume_pairs.cuh"

namespace esdg_vol {

// ---- pipelined persistent kernels -------------------------------------------
// At 160-168 registers per thread one CTA fills an SM, so global-load latency
// in a tile's prologue and epilogue would leave the SM idle.  Here one CTA per
// SM walks its tiles; during tile t's pair pass the copy engine brings the next
// tile's state, geometry (and background) into shared memory (RAW) and tile
// t's own dq (and background right-hand side) (CUR), as 1-D bulk copies
// completing on two mbarriers.  One thread with no pencil issues every copy:
// the 16-byte-aligned interior of each block in bulk and its few unaligned
// edge elements with cp.async.  Tiles come from one mesh (SINGLE: tile t is
// elements t*EPB ..) or from a device work table of (member, first element)
// entries over member descriptors (TABLE: the batched server).  In TABLE mode
// each tile's descriptor is bulk-copied into one of two shared slots with its
// RAW data.  The arithmetic is that of volume_tile, in the same order.
#define ESDG_WAIT_LIMIT (1u << 18)  // polls; about 1 s on GB300
// set when a bounded wait of a pipelined kernel ran out (one flag per
// translation unit; read and cleared through es_dg_sync)
static __device__ int g_esdg_vol_timeout;
static_assert(sizeof(EsdgMember) % 16 == 0, "descriptors are bulk-copied");
// Leaving a CTA on a timeout.  A timeout of the first barrier (this tile's
// data) happens before any other copy of the tile is issued.  A timeout of the
// second (this tile's dq) happens after the next tile's bulk copies were issued
// on the first barrier; they may still be landing in this CTA's shared memory,
// so one thread waits for them (bounded, the same limit) before the CTA exits
// and its shared memory can be handed to another CTA.  The issuing lanes'
// cp.async tails were already waited for before the second barrier.
__device__ __forceinline__ void pipe_drain(unsigned long long* bar, unsigned parity, bool issued) {
  if (issued) esdg_mbar_wait(bar, parity, ESDG_WAIT_LIMIT);
}
// dynamic shared memory a pipelined tile may use (227 KB less static use)
#define ESDG_PIPE_SMEM_MAX (232448 - 1024)

// Tile shape of the pipelined kernels: elements per tile (EPB) and the CTAs
// the launch bounds plan per SM (MINB).  With MINB = 2 two CTAs share an SM,
// so one CTA's FP64 prologue and epilogue run under the other's pair pass; at
// N = 4 two CTAs of 2-element tiles time the same as one CTA of 5-element
// tiles (fewer warps, more idle lanes), and 3-element tiles (8 warps, no
// register spills) are 8 % slower, so the default stays EPB = 5, MINB = 1.
#ifndef ESDG_PIPE4_EPB64
#define ESDG_PIPE4_EPB64 5
#endif
#ifndef ESDG_PIPE4_MINB64
#define ESDG_PIPE4_MINB64 1
#endif
#ifndef ESDG_PIPE4_EPB32
#define ESDG_PIPE4_EPB32 5
#endif
#ifndef ESDG_PIPE4_MINB32
#define ESDG_PIPE4_MINB32 1
#endif
template <int N, bool MIXED>
struct PipeCfg {
  static constexpr int EPB = Cfg<N, MIXED>::EPB, MINB = 1;
};
template <>
struct PipeCfg<4, false> {
  static constexpr int EPB = ESDG_PIPE4_EPB64, MINB = ESDG_PIPE4_MINB64;
};
template <>
struct PipeCfg<4, true> {
  static constexpr int EPB = ESDG_PIPE4_EPB32, MINB = ESDG_PIPE4_MINB32;
};
// the pipelined kernels' Shape (the mixed one carries the background fields)
template <int N, bool MIXED>
using PipeShape = Shape<N, MIXED, MIXED, PipeCfg<N, MIXED>::EPB>;

// The tile with index t: (member, first element, elements).  TABLE: from the
// work table (EPB elements, fewer at a member's end).  SINGLE: EPB-element
// tiles up to tile t1, then tiles of s1 elements, so that the last partial
// round of the persistent grid is spread over all CTAs instead of a few.
template <bool TABLE, int EPB>
__device__ __forceinline__ int4 pipe_tile(const int2* tiles, int t, int t1, int s1, int E) {
  int e0, ne;
  if constexpr (TABLE) {
    const int2 tr = tiles[t];
    return make_int4(tr.x, tr.y, min(EPB, E - tr.y), 0);
  } else {
    if (t < t1) {
      e0 = t * EPB;
      ne = EPB;
    } else {
      e0 = t1 * EPB + (t - t1) * s1;
      ne = s1;
    }
    return make_int4(0, e0, min(ne, E - e0), 0);
  }
}

// Shared state of a pipelined CTA: mbarriers, the tile's (member, e0) in two
// slots, and (TABLE) the member descriptors in two slots.
template <bool TABLE>
struct PipeCtl {
  unsigned long long bars[2];  // [0] RAW of the next tile, [1] CUR of this tile
  int4 info[2];  // (member, first element, elements)
  EsdgMember desc[TABLE ? 2 : 1];
};

template <int N, int MODE>
struct Pipe64 {
  using SH = PipeShape<N, false>;
  static constexpr int P = SH::NP * SH::EPB;  // nodes per tile
  static constexpr int even(int x) { return (x + 1) & ~1; }
  // offsets in doubles, all even (16-byte aligned); each copy target holds
  // four extra doubles for the aligned span around its block
  static constexpr int RAW_Q = 0;                            // [el][5][NP]   next tile's q
  static constexpr int RAW_G = even(RAW_Q + 5 * P + 4);      // [el][11][NP]  next tile's geometry
  static constexpr int S0 = even(RAW_G + ESDG_NVGEO * P + 4);  // [el][18][NP] primitives, Ja/2; exchange
  static constexpr int EPI = even(S0 + SH::NF * P);          // [el][6][NP]   q and 1/J of this tile
  static constexpr int DQ = even(EPI + 6 * P);               // [el][5][NP]   dq of this tile
  static constexpr int TOTAL = MODE ? DQ + 5 * P + 4 : DQ;
  static constexpr size_t SMEM = sizeof(double) * (size_t)TOTAL;
  static_assert(SH::NF == 18, "FP64 node fields");
};

// One block copy of a tile: n elements (4 or 8 bytes) at src, an array that
// ends at lim, into shared memory at dst + sh with sh = (src mod 16)/size.  The
// bulk copy covers the 16-byte-aligned span enclosing the block (it reads up
// to 15 bytes before and after the block, all inside the array: array bases
// are 256-byte aligned allocations or interior pointers of them); only a block
// whose aligned end would pass lim copies its last elements with cp.async.
// dst must be 16-byte aligned with room for n + 2 (16/size) elements.
struct BlockCopy {
  void* dst;
  const void* src;
  const void* lim;
  int n, esz;
};
struct BlockSpan {
  unsigned long long a, b;  // bulk span [a, b)
  int sh, tail0;            // shift; first element copied with cp.async (n if none)
};
__device__ __forceinline__ BlockSpan bc_span(const BlockCopy& c) {
  // element sizes are 4 or 8 bytes: divisions by them are shifts (a 64-bit
  // division by a runtime value costs hundreds of cycles on the issuing lane)
  const unsigned lg = c.esz == 8 ? 3u : 2u;
  const unsigned long long src = reinterpret_cast<unsigned long long>(c.src);
  const unsigned long long end = src + ((unsigned long long)c.n << lg);
  const unsigned long long lim = reinterpret_cast<unsigned long long>(c.lim);
  BlockSpan s;
  s.a = src & ~15ull;
  s.sh = (int)((unsigned)(src - s.a) >> lg);
  const unsigned long long up = (end + 15ull) & ~15ull;
  s.b = up <= lim ? up : (end & ~15ull);
  if (s.b < s.a) s.b = s.a;
  s.tail0 = s.b >= end ? c.n : (s.b > src ? (int)((s.b - src) >> lg) : 0);
  return s;
}

// The copy issue of a pipelined CTA is spread over the lanes that own no pencil
// (all in the last warp; thread 0 alone when every lane has a pencil): lane il
// of nl takes blocks il, il + nl, ...; a warp sum of the lanes' bulk bytes
// (plus an optional extra bulk copy, the next member's descriptor) is
// registered on the barrier before any copy is issued.
template <int T, int PENCILS>
struct Issuers {
  static constexpr bool IDLE = PENCILS < T;
  static constexpr int FIRST = IDLE ? PENCILS : 0;
  static constexpr int COUNT = IDLE ? T - PENCILS : 1;
  static_assert(!IDLE || PENCILS / 32 == (T - 1) / 32, "idle lanes share the last warp");
  static __device__ __forceinline__ unsigned mask() {
    return IDLE ? (0xffffffffu << (PENCILS % 32)) : 1u;
  }
  static __device__ __forceinline__ bool is(int tid) { return tid >= FIRST && tid < FIRST + COUNT; }
};
// phantom: bytes registered but never copied (a test hook that makes the
// barrier's bounded wait run out; 0 in normal operation)
// track_cp: every issuing lane also arrives on the barrier (cp.async.mbarrier
// .arrive.noinc) once its cp.async edge copies have landed, so that threads
// other than the issuers may wait on the barrier alone; the barrier then
// expects 1 + ISS::COUNT arrivals per phase.
template <typename ISS, int MAXB>
__device__ __forceinline__ void pipe_issue(int tid, const BlockCopy (&bl)[MAXB], int nb,
                                           unsigned long long* bar, unsigned extra = 0,
                                           const void* xsrc = nullptr, void* xdst = nullptr,
                                           unsigned phantom = 0, bool track_cp = false) {
  constexpr int PER = (MAXB + ISS::COUNT - 1) / ISS::COUNT;
  const int il = tid - ISS::FIRST;
  BlockSpan sp[PER];
  unsigned mine = 0;
#pragma unroll
  for (int k = 0; k < PER; k++) {
    const int b = il + k * ISS::COUNT;
    if (b < nb && bl[b].n > 0) {
      sp[k] = bc_span(bl[b]);
      mine += (unsigned)(sp[k].b - sp[k].a);
    }
  }
  const unsigned total =
      (ISS::COUNT > 1 ? __reduce_add_sync(ISS::mask(), mine) : mine) + extra + phantom;
  if (il == 0) esdg_mbar_arrive_tx(bar, total);
  if (ISS::COUNT > 1) __syncwarp(ISS::mask());
  esdg_fence_proxy_async();
  if (il == 0 && extra) esdg_bulk_g2s(xdst, xsrc, extra, bar);
#pragma unroll
  for (int k = 0; k < PER; k++) {
    const int b = il + k * ISS::COUNT;
    if (b < nb && bl[b].n > 0) {
      const BlockCopy& c = bl[b];
      if (sp[k].b > sp[k].a)
        esdg_bulk_g2s(c.dst, reinterpret_cast<const void*>(sp[k].a), (unsigned)(sp[k].b - sp[k].a), bar);
      for (int i = sp[k].tail0; i < c.n; i++) {
        if (c.esz == 8)
          esdg_cp_async(static_cast<double*>(c.dst) + sp[k].sh + i, static_cast<const double*>(c.src) + i);
        else
          esdg_cp_async(static_cast<float*>(c.dst) + sp[k].sh + i, static_cast<const float*>(c.src) + i);
      }
    }
  }
  if (track_cp)
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(esdg_smem_addr(bar))
                 : "memory");
}

template <int N, int MODE, bool TABLE>
__global__ void __launch_bounds__(PipeShape<N, false>::THREADS, PipeCfg<N, false>::MINB)
    k_volume_pipe64(const EsdgMember one, const EsdgMember* __restrict__ members,
                    const int2* __restrict__ tiles, const int* __restrict__ ntiles_d, int ntiles_1,
                    EsdgLGL L, double rkA, double rkB, unsigned phantom, int t1, int s1) {
  static_assert(!TABLE || MODE == 1, "the batched kernel applies an RK stage");
  using SH = PipeShape<N, false>;
  using PP = Pipe64<N, MODE>;
  constexpr int Nq = SH::Nq, NP = SH::NP, NPEN = SH::NPEN, EPB = SH::EPB, NF = SH::NF;
  constexpr int T = SH::THREADS;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) PipeCtl<TABLE> ctl;
  double* sm = reinterpret_cast<double*>(smraw);
  const int tid = threadIdx.x;
  const int ntiles = TABLE ? *ntiles_d : ntiles_1;

  using ISS = Issuers<T, SH::PENCILS>;
  // the next tile as seen by the issuing lanes (fetched early: in TABLE mode
  // these are global loads whose latency the prologue hides)
  struct Next {
    int4 tr;  // (member, first element, elements)
    int E;
    const double* q;
    const double* vg;
    const EsdgMember* Mg;
  };
  auto fetch = [&](int t) {
    Next x;
    const int m = TABLE ? tiles[t].x : 0;
    x.Mg = TABLE ? members + m : &ctl.desc[0];
    x.E = x.Mg->g.E;
    x.tr = pipe_tile<TABLE, EPB>(tiles, t, t1, s1, x.E);
    x.q = x.Mg->a.q_in;
    x.vg = reinterpret_cast<const double*>(x.Mg->a.vgeo);
    return x;
  };
  // issuing lanes: the next tile's (member, e0), descriptor and RAW blocks into slot s
  auto issue_next = [&](const Next& x, int s, unsigned ph = 0) {
    if (tid == ISS::FIRST) ctl.info[s] = x.tr;
    const int e0 = x.tr.y, ne = x.tr.z;
    const BlockCopy bl[2] = {
        {sm + PP::RAW_Q, x.q + (size_t)e0 * 5 * NP, x.q + (size_t)x.E * 5 * NP, ne * 5 * NP, 8},
        {sm + PP::RAW_G, x.vg + (size_t)e0 * ESDG_NVGEO * NP, x.vg + (size_t)x.E * ESDG_NVGEO * NP,
         ne * ESDG_NVGEO * NP, 8}};
    if constexpr (TABLE)
      pipe_issue<ISS>(tid, bl, 2, &ctl.bars[0], (unsigned)sizeof(EsdgMember), x.Mg, &ctl.desc[s], ph);
    else
      pipe_issue<ISS>(tid, bl, 2, &ctl.bars[0], 0, nullptr, nullptr, ph);
  };

  if (tid == 0) {
    esdg_mbar_init(&ctl.bars[0], 1);
    esdg_mbar_init(&ctl.bars[1], 1);
    esdg_fence_mbar_init();
    if constexpr (!TABLE) ctl.desc[0] = one;
  }
  __syncthreads();
  if (ISS::is(tid) && (int)blockIdx.x < ntiles) issue_next(fetch(blockIdx.x), 0, phantom);
  unsigned ph_raw = 0, ph_cur = 0;
  int slot = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, slot ^= 1) {
    esdg_cp_async_wait_all();  // this lane's tail copies
    const bool ok = esdg_mbar_wait(&ctl.bars[0], ph_raw, ESDG_WAIT_LIMIT);
    ph_raw ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
      return;
    }
    const EsdgMember& M = ctl.desc[TABLE ? slot : 0];
    const EsdgGrid& g = M.g;
    const EsdgPhys& P = M.P;
    const EsdgVolArgs& a = M.a;
    const int E = g.E, e0 = ctl.info[slot].y, ne = ctl.info[slot].z;
    const int next = tile + (int)gridDim.x;
    // issuing lanes: this tile's dq (CUR) now, the next tile's location early
    Next nx;
    if (ISS::is(tid)) {
      if constexpr (MODE != 0) {
        const double* dqg = reinterpret_cast<const double*>(a.dq);
        const BlockCopy cb[1] = {{sm + PP::DQ, dqg + (size_t)e0 * 5 * NP, dqg + (size_t)E * 5 * NP,
                                  ne * 5 * NP, 8}};
        pipe_issue<ISS>(tid, cb, 1, &ctl.bars[1]);
      }
      if (TABLE && next < ntiles) nx = fetch(next);  // global loads: early
    }
    // ---- prologue: RAW -> primitives, Ja/2 (S) and q, 1/J (EPI) -----------
    {
      const double* vg = reinterpret_cast<const double*>(a.vgeo);
      const double* qr0 = sm + PP::RAW_Q + esdg_block_shift(a.q_in + (size_t)e0 * 5 * NP);
      const double* gr0 = sm + PP::RAW_G + esdg_block_shift(vg + (size_t)e0 * ESDG_NVGEO * NP);
      const double gm1 = P.gamma - 1.0;
      for (int idx = tid; idx < EPB * NP; idx += T) {
        const int el2 = idx / NP, n = idx - el2 * NP;
        double* S = sm + PP::S0 + (size_t)el2 * NF * NP;
        if (el2 < ne) {
          const double* qr = qr0 + (size_t)el2 * 5 * NP;
          const double* gr = gr0 + (size_t)el2 * ESDG_NVGEO * NP;
          double* X = sm + PP::EPI + (size_t)el2 * 6 * NP;
          const double q0 = qr[n], q1 = qr[NP + n], q2 = qr[2 * NP + n], q3 = qr[3 * NP + n],
                       q4 = qr[4 * NP + n];
          prims64<NP>(q0, q1, q2, q3, q4, gr[10 * NP + n], gm1, S, n);
#pragma unroll
          for (int k = 0; k < 9; k++) S[(SH::F_NH + k) * NP + n] = gr[k * NP + n];
          X[n] = q0;
          X[NP + n] = q1;
          X[2 * NP + n] = q2;
          X[3 * NP + n] = q3;
          X[4 * NP + n] = q4;
          // 1/J, times dt for a stage update (the epilogue's scale)
          X[5 * NP + n] = MODE != 0 ? gr[9 * NP + n] * a.dt : gr[9 * NP + n];
        } else {  // padding element: any valid state, results are discarded
          S[0 * NP + n] = 0.25;
          S[1 * NP + n] = 0.5;
          S[2 * NP + n] = 1.0;
          for (int k = 3; k < NF; k++) S[k * NP + n] = 0.0;
        }
      }
    }
    __syncthreads();  // RAW consumed

    int need_logs = 0;
    for (int idx = tid; idx < EPB * NP; idx += T) {
      const int el2 = idx / NP, n = idx - el2 * NP;
      if (out_of_series64<NP>(sm + PP::S0 + (size_t)el2 * NF * NP, n)) need_logs = 1;
    }
    need_logs = __syncthreads_or(need_logs);
    if (need_logs) {
      for (int idx = tid; idx < EPB * NP; idx += T) {
        const int el2 = idx / NP, n = idx - el2 * NP;
        double* S = sm + PP::S0 + (size_t)el2 * NF * NP;
        S[SH::F_LR * NP + n] = log(4.0 * S[n]);
        S[SH::F_LB * NP + n] = log(2.0 * S[NP + n]);
      }
      __syncthreads();
    }
    // the copies for this tile's epilogue and the next tile
    if (ISS::is(tid) && next < ntiles) issue_next(TABLE ? nx : fetch(next), slot ^ 1);

    // ---- pair pass: this thread's pencil (index arithmetic redone per tile
    // rather than held in registers across the pair pass) -------------------
    const bool active = tid < SH::PENCILS;
    const int el = active ? tid / (3 * NPEN) : 0;
    const int rr = tid - el * 3 * NPEN;
    const int d = active ? rr / NPEN : 0;
    const int pen = rr - d * NPEN;
    const int ps = pen % Nq, pt = pen / Nq;
    const int stride = (d == 0) ? 1 : ((d == 1) ? Nq : Nq * Nq);
    const int base = (d == 0) ? Nq * (ps + Nq * pt) : ((d == 1) ? (ps + Nq * Nq * pt) : (ps + Nq * pt));
    const int e = e0 + el;
    double acc[Nq][5];
#pragma unroll
    for (int i = 0; i < Nq; i++)
#pragma unroll
      for (int v = 0; v < 5; v++) acc[i][v] = 0.0;
    if (active && el < ne) {
      face_lift<true, N, double>(g, a, e, d, ps + Nq * pt, acc);
      const double* S = sm + PP::S0 + (size_t)el * NF * NP;
      if (need_logs)
        pencil_pass<N, false, true, false>(S, d, base, stride, L, ce_series(0.5 * P.igm1), acc);
      else
        pencil_pass<N, false, false, false>(S, d, base, stride, L, ce_series(0.5 * P.igm1), acc);
    }
    __syncthreads();
    if (active && el < ne) {
      double* S = sm + PP::S0 + (size_t)el * NF * NP;
#pragma unroll
      for (int i = 0; i < Nq; i++)
#pragma unroll
        for (int v = 0; v < 5; v++) S[(d * 5 + v) * NP + base + i * stride] = acc[i][v];
    }
    if constexpr (MODE != 0) {
      esdg_cp_async_wait_all();
      const bool okd = esdg_mbar_wait(&ctl.bars[1], ph_cur, ESDG_WAIT_LIMIT);  // this tile's dq
      ph_cur ^= 1u;
      if (__syncthreads_or(!okd)) {
        if (tid == 0) {
          atomicExch(&g_esdg_vol_timeout, 1);
          pipe_drain(&ctl.bars[0], ph_raw, next < ntiles);
        }
        return;
      }
    } else {
      __syncthreads();
    }

    // ---- epilogue: one thread per (node, variable) (eight full rounds instead
    // of one and a partial one per node) ---------------------------------------
    const double* D0 = sm + PP::DQ + esdg_block_shift(reinterpret_cast<const double*>(a.dq) + (size_t)e0 * 5 * NP);
    // descriptor fields in registers (the stores below would force reloads)
    const double dt = a.dt;
    const EsdgPhys Pl = P;
    const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
    const double* xg = a.x;
    double* const dqp = reinterpret_cast<double*>(a.dq);
    double* const qio = a.q_io;
    double* const rhsp = a.rhs;
    int* const status = a.status;
    bool bad = false;
    for (int idx = tid; idx < 5 * EPB * NP; idx += T) {
      const int v = idx / (EPB * NP), rem = idx - v * (EPB * NP);
      const int el2 = rem / NP, n = rem - el2 * NP, e2 = e0 + el2;
      if (el2 >= ne) continue;
      const double* S = sm + PP::S0 + (size_t)el2 * NF * NP;
      const double* X = sm + PP::EPI + (size_t)el2 * 6 * NP;
      double r = -X[5 * NP + n] * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
      if (rot && (v == 1 || v == 2)) {
        const double y = xg[((size_t)e2 * 3 + 1) * NP + n];
        double f = Pl.f0 + Pl.beta * (y - Pl.y0);
        if constexpr (MODE != 0) f *= dt;
        r = v == 1 ? fma(f, X[2 * NP + n], r) : fma(-f, X[NP + n], r);
      }
      const size_t qv = ((size_t)e2 * 5 + v) * NP + n;
      if constexpr (MODE == 0) {
        rhsp[qv] = r;
      } else {
        // first stage (A = 0): the register is not read (see stage32)
        const double dv = rkA == 0.0 ? r : fma(rkA, D0[((size_t)el2 * 5 + v) * NP + n], r);
        dqp[qv] = dv;
        const double qn = fma(rkB, dv, X[v * NP + n]);
        qio[qv] = qn;
        bad |= esdg_bad_state(qn, v == 0);
      }
    }
    if (MODE != 0 && bad && status) *status = 1;
  }
}

// ---- pipelined persistent mixed-precision kernel (with a background) ------
template <int N, int MODE>
struct Pipe32 {
  using SH = PipeShape<N, true>;
  static constexpr int NP = SH::NP, EPB = SH::EPB, P = NP * EPB;
  static constexpr int up16(int b) { return (b + 15) & ~15; }
  // byte offsets, 16-byte aligned; copy targets hold 32 extra bytes (the
  // aligned span around each block)
  static constexpr int RAW_Q = 0;                                  // [el][5][NP]  double
  static constexpr int RAW_BG = up16(RAW_Q + 8 * (5 * P + 4));     // [el][3][NP]  double rho_bg, E_bg, phi
  static constexpr int RAW_BGP = up16(RAW_BG + 8 * (3 * P + 4));   // [el][4][NP]  float background fields
  static constexpr int RAW_G = up16(RAW_BGP + 4 * (4 * P + 8));    // [el][11][NP] float
  static constexpr int S0 = up16(RAW_G + 4 * (ESDG_NVGEO * P + 8));  // [el][NF][NP] float
  static constexpr int EPI_Q = up16(S0 + 4 * SH::NF * P);         // [el][5][NP]  double
  static constexpr int EPI_J = up16(EPI_Q + 8 * 5 * P);           // [el][NP]     float
  static constexpr int CUR_RB = up16(EPI_J + 4 * P);              // [el][3][NP]  float
  static constexpr int CUR_DQ = up16(CUR_RB + 4 * (3 * P + 8));   // [el][5][NP]  float
  static constexpr int TOTAL = MODE ? up16(CUR_DQ + 4 * (5 * P + 8)) : CUR_DQ;
  static constexpr size_t SMEM = (size_t)TOTAL;
};

template <int N, int MODE, bool TABLE>
__global__ void __launch_bounds__(PipeShape<N, true>::THREADS, PipeCfg<N, true>::MINB)
    k_volume_pipe32(const EsdgMember one, const EsdgMember* __restrict__ members,
                    const int2* __restrict__ tiles, const int* __restrict__ ntiles_d, int ntiles_1,
                    EsdgLGL L, double rkA, double rkB, unsigned phantom, int t1, int s1) {
  static_assert(!TABLE || MODE == 1, "the batched kernel applies an RK stage");
  using SH = PipeShape<N, true>;
  using PP = Pipe32<N, MODE>;
  constexpr int Nq = SH::Nq, NP = SH::NP, NPEN = SH::NPEN, EPB = SH::EPB, NF = SH::NF;
  constexpr int T = SH::THREADS;
  constexpr int NN = EPB * NP;  // nodes of a tile
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) PipeCtl<TABLE> ctl;
  __shared__ float phi0s[EPB];  // each element's reference geopotential
  double* const rawq = reinterpret_cast<double*>(smraw + PP::RAW_Q);
  double* const rawbg = reinterpret_cast<double*>(smraw + PP::RAW_BG);
  float* const rawbgp = reinterpret_cast<float*>(smraw + PP::RAW_BGP);
  float* const rawg = reinterpret_cast<float*>(smraw + PP::RAW_G);
  float* const sm = reinterpret_cast<float*>(smraw + PP::S0);
  double* const epq = reinterpret_cast<double*>(smraw + PP::EPI_Q);
  float* const epj = reinterpret_cast<float*>(smraw + PP::EPI_J);
  float* const currb = reinterpret_cast<float*>(smraw + PP::CUR_RB);
  float* const curdq = reinterpret_cast<float*>(smraw + PP::CUR_DQ);
  const int tid = threadIdx.x;
  const int ntiles = TABLE ? *ntiles_d : ntiles_1;

  using ISS = Issuers<T, SH::PENCILS>;
  struct Next {
    int4 tr;  // (member, first element, elements)
    int E;
    const double* q;
    const double* bg;
    const float* bgp;
    const float* vg;
    const EsdgMember* Mg;
  };
  auto fetch = [&](int t) {
    Next x;
    const int m = TABLE ? tiles[t].x : 0;
    x.Mg = TABLE ? members + m : &ctl.desc[0];
    x.E = x.Mg->g.E;
    x.tr = pipe_tile<TABLE, EPB>(tiles, t, t1, s1, x.E);
    x.q = x.Mg->a.q_in;
    x.bg = x.Mg->a.bg;
    x.bgp = x.Mg->a.bgp;
    x.vg = reinterpret_cast<const float*>(x.Mg->a.vgeo);
    return x;
  };
  // issuing lanes: the next tile's (member, e0), descriptor and RAW blocks into slot s
  auto issue_next = [&](const Next& x, int s, unsigned ph = 0) {
    if (tid == ISS::FIRST) ctl.info[s] = x.tr;
    const int e0 = x.tr.y, ne = x.tr.z;
    const BlockCopy bl[4] = {
        {rawq, x.q + (size_t)e0 * 5 * NP, x.q + (size_t)x.E * 5 * NP, ne * 5 * NP, 8},
        {rawbg, x.bg + (size_t)e0 * 3 * NP, x.bg + (size_t)x.E * 3 * NP, ne * 3 * NP, 8},
        {rawbgp, x.bgp + (size_t)e0 * 4 * NP, x.bgp + (size_t)x.E * 4 * NP, ne * 4 * NP, 4},
        {rawg, x.vg + (size_t)e0 * ESDG_NVGEO * NP, x.vg + (size_t)x.E * ESDG_NVGEO * NP,
         ne * ESDG_NVGEO * NP, 4}};
    if constexpr (TABLE)
      pipe_issue<ISS>(tid, bl, 4, &ctl.bars[0], (unsigned)sizeof(EsdgMember), x.Mg, &ctl.desc[s], ph);
    else
      pipe_issue<ISS>(tid, bl, 4, &ctl.bars[0], 0, nullptr, nullptr, ph);
  };

  if (tid == 0) {
    esdg_mbar_init(&ctl.bars[0], 1);
    esdg_mbar_init(&ctl.bars[1], 1);
    esdg_fence_mbar_init();
    if constexpr (!TABLE) ctl.desc[0] = one;
  }
  __syncthreads();
  if (ISS::is(tid) && (int)blockIdx.x < ntiles) issue_next(fetch(blockIdx.x), 0, phantom);
  unsigned ph_raw = 0, ph_cur = 0;
  int slot = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, slot ^= 1) {
    esdg_cp_async_wait_all();  // this lane's tail copies
    const bool ok = esdg_mbar_wait(&ctl.bars[0], ph_raw, ESDG_WAIT_LIMIT);
    ph_raw ^= 1u;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
      return;
    }
    const EsdgMember& M = ctl.desc[TABLE ? slot : 0];
    const EsdgGrid& g = M.g;
    const EsdgPhys& P = M.P;
    const EsdgVolArgs& a = M.a;
    const int E = g.E, e0 = ctl.info[slot].y, ne = ctl.info[slot].z;
    const int next = tile + (int)gridDim.x;
    // issuing lanes: this tile's background rhs and dq (CUR) now, the next
    // tile's location early
    Next nx;
    if (ISS::is(tid)) {
      const float* dqg = reinterpret_cast<const float*>(a.dq);
      const BlockCopy cb[2] = {
          {currb, a.rhs_bg + (size_t)e0 * 3 * NP, a.rhs_bg + (size_t)E * 3 * NP, ne * 3 * NP, 4},
          {curdq, dqg + (size_t)e0 * 5 * NP, dqg + (size_t)E * 5 * NP, MODE ? ne * 5 * NP : 0, 4}};
      pipe_issue<ISS>(tid, cb, 2, &ctl.bars[1]);
      if (TABLE && next < ntiles) nx = fetch(next);  // global loads: early
    }
    // ---- prologue, two nodes per thread and round (their FP64 chains and
    // loads interleave; descriptor fields held in registers: the shared-memory
    // stores below would otherwise force their reloads) ----------------------
    {
      const float gm1f = esdg_d2f(P.gamma - 1.0);
      const float* vg = reinterpret_cast<const float*>(a.vgeo);
      const double* qr0 = rawq + esdg_block_shift(a.q_in + (size_t)e0 * 5 * NP);
      const double* br0 = rawbg + esdg_block_shift(a.bg + (size_t)e0 * 3 * NP);
      const float* pr0 = rawbgp + esdg_block_shift(a.bgp + (size_t)e0 * 4 * NP);
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
          if (n == 0) phi0s[el] = esdg_d2f(x.phi);
        } else {  // padding element: any valid state, results are discarded
          S[0 * NP + n] = 0.25f;
          S[1 * NP + n] = 0.5f;
          S[2 * NP + n] = 1.0f;
          for (int f = 3; f < NF; f++) S[f * NP + n] = 0.0f;
        }
      };
      auto prim = [&](const In& x) {
        return prims32bg(x.q0, x.q1, x.q2, x.q3, x.q4, x.phi, x.phh, gm1f, x.rb, x.eb, x.b0, x.b1,
                         x.b2, x.b3);
      };
      // two nodes per thread and round; a warp whose second slots all lie
      // past the tile (warp-uniform test on its first lane) converts one
      for (int i0 = tid; i0 < NN; i0 += 2 * T) {
        if (i0 - (tid & 31) + T < NN) {
          const In x0 = load(i0), x1 = load(i0 + T);
          const Prim32 o0 = prim(x0), o1 = prim(x1);
          store(x0, o0);
          store(x1, o1);
        } else {
          const In x0 = load(i0);
          store(x0, prim(x0));
        }
      }
    }
    __syncthreads();  // RAW consumed

    int need_logs = 0;
    for (int idx = tid; idx < NN; idx += T) {
      const int el2 = idx / NP, n = idx - el2 * NP;
      const float* S = sm + (size_t)el2 * NF * NP;
      const float r0 = S[0], rn = S[n], b0 = S[NP], bn = S[NP + n];
      // |f| < 0.14 keeps u < ESDG_LOG_EPS32 for every pair
      if (fabsf(rn - r0) > 0.13f * r0 || fabsf(bn - b0) > 0.13f * b0) need_logs = 1;
    }
    need_logs = __syncthreads_or(need_logs);
    // the copies for this tile's epilogue and the next tile
    if (ISS::is(tid) && next < ntiles) issue_next(TABLE ? nx : fetch(next), slot ^ 1);

    // ---- pair pass ------------------------------------------------------------
    const bool active = tid < SH::PENCILS;
    const int el = active ? tid / (3 * NPEN) : 0;
    const int rr = tid - el * 3 * NPEN;
    const int d = active ? rr / NPEN : 0;
    const int pen = rr - d * NPEN;
    const int ps = pen % Nq, pt = pen / Nq;
    const int stride = (d == 0) ? 1 : ((d == 1) ? Nq : Nq * Nq);
    const int base = (d == 0) ? Nq * (ps + Nq * pt) : ((d == 1) ? (ps + Nq * Nq * pt) : (ps + Nq * pt));
    const int e = e0 + el;
    float acc[Nq][5];
#pragma unroll
    for (int i = 0; i < Nq; i++)
#pragma unroll
      for (int v = 0; v < 5; v++) acc[i][v] = 0.0f;
    if (active && el < ne) {
      const FaceTerms<float> ft = face_fetch<N, float>(g, a, e, d, ps + Nq * pt);
      const float* S = sm + (size_t)el * NF * NP;
      const float ce = esdg_d2f(0.5 * P.igm1);
      if (need_logs)
        pencil_pass<N, true, true, true>(S, d, base, stride, L, ce, acc);
      else
        pencil_pass<N, true, false, true>(S, d, base, stride, L, ce, acc);
      const float phi0 = phi0s[el];
#pragma unroll
      for (int i = 0; i < Nq; i++) acc[i][4] = fmaf(phi0, acc[i][0], acc[i][4]);
      face_add<N, float>(ft, acc);
    }
    __syncthreads();
    if (active && el < ne) {
      float* S = sm + (size_t)el * NF * NP;
#pragma unroll
      for (int i = 0; i < Nq; i++)
#pragma unroll
        for (int v = 0; v < 5; v++) S[(d * 5 + v) * NP + base + i * stride] = acc[i][v];
    }
    esdg_cp_async_wait_all();
    const bool okc = esdg_mbar_wait(&ctl.bars[1], ph_cur, ESDG_WAIT_LIMIT);
    ph_cur ^= 1u;
    if (__syncthreads_or(!okc)) {
      if (tid == 0) {
        atomicExch(&g_esdg_vol_timeout, 1);
        pipe_drain(&ctl.bars[0], ph_raw, next < ntiles);
      }
      return;
    }

    // ---- epilogue, two nodes per thread and round ------------------------------
    const float* RB0 = currb + esdg_block_shift(a.rhs_bg + (size_t)e0 * 3 * NP);
    const float* D0 = curdq + esdg_block_shift(reinterpret_cast<const float*>(a.dq) + (size_t)e0 * 5 * NP);
    const EsdgPhys Pl = P;
    const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
    const double* xg = a.x;
    float* const dqp = reinterpret_cast<float*>(a.dq);
    double* const qio = a.q_io;
    double* const rhsp = a.rhs;
    const double dtv = a.dt;
    int* const status = a.status;
    bool bad = false;
    for (int i0 = tid; i0 < NN; i0 += 2 * T) {
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const int idx = i0 + k * T;
        const int el2 = idx / NP, n = idx - el2 * NP, e2 = e0 + el2;
        if (idx >= NN || el2 >= ne) continue;
        const float* S = sm + (size_t)el2 * NF * NP;
        const double* X = epq + (size_t)el2 * 5 * NP;
        const float iJ = epj[(size_t)el2 * NP + n];
        const float* RB = RB0 + (size_t)el2 * 3 * NP;
        const size_t qb = (size_t)e2 * 5 * NP + n;
        if constexpr (MODE != 0) {
          float r32[5];
#pragma unroll
          for (int v = 0; v < 5; v++)
            r32[v] = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
          const double y = rot ? xg[((size_t)e2 * 3 + 1) * NP + n] : 0.0;
          bad |= stage32<NP, true>(r32, RB + n, Pl, y, X + n, D0 + (size_t)el2 * 5 * NP + n,
                                   dqp + qb, qio + qb, rkA, rkB, dtv);
        } else {  // right-hand side in FP64
          double r[5];
#pragma unroll
          for (int v = 0; v < 5; v++) {
            const float rv = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
            r[v] = esdg_f2d(rv + (v >= 1 && v <= 3 ? RB[(v - 1) * NP + n] : 0.0f));
          }
          if (rot) {
            const double y = xg[((size_t)e2 * 3 + 1) * NP + n];
            const double f = Pl.f0 + Pl.beta * (y - Pl.y0);
            r[1] = fma(f, X[2 * NP + n], r[1]);
            r[2] = fma(-f, X[NP + n], r[2]);
          }
#pragma unroll
          for (int v = 0; v < 5; v++) rhsp[qb + (size_t)v * NP] = r[v];
        }
      }
    }
    if (MODE != 0 && bad && status) *status = 1;
  }
}

// Launch helpers: the resident CTAs per device are found once per kernel
// (the cache is keyed on the kernel itself, a template argument)
template <auto k>
int pipe_grid_cap(int threads, size_t smem) {
  constexpr int MAXDEV = 64;
  static int cap[MAXDEV];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return -1;
  if (cap[dev] == 0) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return -1;
    int per_sm = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
      return -1;
    cap[dev] = per_sm * nsm;
  }
  return cap[dev];
}

// Tiles of a single mesh of E elements on a persistent grid of at most cap
// CTAs: full rounds of EPB-element tiles, then the remaining elements as tiles
// of s1 = ceil(rest / cap) elements, so the last round is spread over the grid.
inline void pipe_split(int E, int EPB, int cap, int& ntiles, int& grid, int& t1, int& s1) {
  const int nfull = (E + EPB - 1) / EPB;
  grid = nfull < cap ? nfull : cap;
  if (grid <= 0) {
    ntiles = grid = t1 = 0;
    s1 = 1;
    return;
  }
  t1 = (nfull / grid) * grid;  // tiles of the full rounds
  if (t1 * EPB >= E) {         // no partial round
    t1 = nfull;
    s1 = EPB;
    ntiles = nfull;
    return;
  }
  const int rest = E - t1 * EPB;
  s1 = (rest + grid - 1) / grid;
  ntiles = t1 + (rest + s1 - 1) / s1;
}

inline EsdgMember pipe_member(const EsdgGrid& g, const EsdgPhys& P, const EsdgVolArgs& a) {
  EsdgMember m;
  memset(&m, 0, sizeof(m));
  m.g = g;
  m.P = P;
  m.a = a;
  m.bg = a.bg;
  return m;
}

template <int N, int MODE>
cudaError_t launch_pipe64(const EsdgGrid& g, const EsdgPhys& P, const EsdgLGL& L,
                          const EsdgVolArgs& a, cudaStream_t s) {
  using SH = PipeShape<N, false>;
  constexpr auto k = k_volume_pipe64<N, MODE, false>;
  const int cap = pipe_grid_cap<k>(SH::THREADS, Pipe64<N, MODE>::SMEM);
  if (cap < 0) return cudaErrorInvalidConfiguration;
  int ntiles, grid, t1, s1;
  pipe_split(g.E, SH::EPB, cap, ntiles, grid, t1, s1);
  if (ntiles == 0) return cudaSuccess;
  k<<<grid, SH::THREADS, Pipe64<N, MODE>::SMEM, s>>>(pipe_member(g, P, a), nullptr, nullptr, nullptr,
                                                     ntiles, L, a.rkA, a.rkB, esdg_take_phantom(),
                                                     t1, s1);
  return cudaGetLastError();
}

template <int N, int MODE>
cudaError_t launch_pipe32(const EsdgGrid& g, const EsdgPhys& P, const EsdgLGL& L,
                          const EsdgVolArgs& a, cudaStream_t s) {
  using SH = PipeShape<N, true>;
  constexpr auto k = k_volume_pipe32<N, MODE, false>;
  const int cap = pipe_grid_cap<k>(SH::THREADS, Pipe32<N, MODE>::SMEM);
  if (cap < 0) return cudaErrorInvalidConfiguration;
  int ntiles, grid, t1, s1;
  pipe_split(g.E, SH::EPB, cap, ntiles, grid, t1, s1);
  if (ntiles == 0) return cudaSuccess;
  k<<<grid, SH::THREADS, Pipe32<N, MODE>::SMEM, s>>>(pipe_member(g, P, a), nullptr, nullptr, nullptr,
                                                     ntiles, L, a.rkA, a.rkB, esdg_take_phantom(),
                                                     t1, s1);
  return cudaGetLastError();
}

// batched (TABLE) launches; what: 0 launch (0 / -1), 1 elements per tile, 2 CTAs per SM
template <int N, bool MIXED>
int pipe_batch(int what, const EsdgMember* members, const int2* tiles, const int* ntiles, int grid,
               const EsdgLGL& L, double A, double B, cudaStream_t s) {
  using SH = PipeShape<N, MIXED>;
  constexpr size_t SMEM = MIXED ? Pipe32<N, 1>::SMEM : Pipe64<N, 1>::SMEM;
  if (what == 1) return SH::EPB;
  auto k = [] {
    if constexpr (MIXED) return k_volume_pipe32<N, 1, true>;
    else return k_volume_pipe64<N, 1, true>;
  }();
  if (what == 2) {
    int nb = 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, SH::THREADS, SMEM) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    return nb > 0 ? nb : 1;
  }
  static bool configured = false;  // one-time attribute set per instantiation
  if (!configured) {
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM) != cudaSuccess)
      return -1;
    configured = true;
  }
  EsdgMember none;
  memset(&none, 0, sizeof(none));
  k<<<grid, SH::THREADS, SMEM, s>>>(none, members, tiles, ntiles, 0, L, A, B, 0u, 0, 0);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace esdg_vol
