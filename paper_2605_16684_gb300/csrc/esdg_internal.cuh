// esdg_internal.cuh -- device-side definitions shared by the library's kernels.
//
// Data layout in HBM (one handle, E elements, np = Nq^3 nodes each):
//   q, dq, rhs      double [E][5][np]            element-major, variable, node
//   vgeo            double [E][11][np]           1/2 Ja^d_c (9), 1/J, phi
//   vgeo32          float  [E][11][np]           same, FP32 copy (mixed mode)
//   x               double [E][3][np]            node coordinates
//   fgeo            double [F][5][Nq^2]          nhat (3), s / w_end, phi per face node
//   fflux           double/float [F][5][Nq^2]    (s / w_end) F* per face node
// Faces are numbered direction by direction: face (d, P, a, b) with plane P along
// d and element indices (a, b) along the two other directions in increasing
// order; its node (s, t) has node index s along the first, t along the second.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#define ESDG_NV 5
#define ESDG_MAXNQ 8
#define ESDG_NVGEO 11

struct EsdgLGL {  // LGL operators, passed by value (lives in the constant bank)
  int N;
  double xi[ESDG_MAXNQ];
  double w[ESDG_MAXNQ];
  double D[ESDG_MAXNQ][ESDG_MAXNQ];   // nodal differentiation matrix
  double Dt[ESDG_MAXNQ][ESDG_MAXNQ];  // 2D - W^-1 B, zero diagonal
  float Dtf[ESDG_MAXNQ][ESDG_MAXNQ];  // FP32 copy for the mixed-precision pair loop
  double xi_lo[ESDG_MAXNQ];           // low parts (xi = xi + xi_lo, D = D + D_lo) for the
  double D_lo[ESDG_MAXNQ][ESDG_MAXNQ];  // double-double geometry construction
};

struct EsdgPhys {
  double gamma, g, R, p0, f0, beta, y0;
  int dissipation;
  double igm1, igamma;  // 1/(gamma-1) and 1/gamma, set by esdg_phys_derive on the host
};
inline void esdg_phys_derive(EsdgPhys* P) {
  P->igm1 = 1.0 / (P->gamma - 1.0);
  P->igamma = 1.0 / P->gamma;
}

struct EsdgGrid {  // structured box and derived face numbering
  int K[3];
  int periodic[3];
  double lo[3], hi[3];  // the whole box (a partition keeps its parent's)
  double warp;
  int N, Nq, np, E;
  int nplanes[3];
  long long face_off[3];
  long long nfaces;
  // A partition of a larger box: its elements are the parent's elements
  // eoff + (0..K-1) of Kg per direction (node positions follow from the parent
  // mesh), and remote[0] / remote[1] mark its low / high x plane as a cut whose
  // outside state arrives as a trace from the neighbouring partition.  A whole
  // mesh has eoff = 0, Kg = K, remote = 0.
  int eoff[3], Kg[3];
  int remote[2];
};

// Outside states of a partition's remote x planes, [face in plane][nv][Nq^2]
// with the plane's faces in face-id order: slots 0-4 the conserved state, and
// for mixed-precision handles slots 5-6 the background rho_bg and p_bg of the
// same node (nv = 7).  bgmode = 1 makes the outside state the background at
// rest (rho_bg, 0, 0, 0, p_bg/(gamma-1) + rho_bg phi), for the background's own
// right-hand side.  Null pointers: no remote plane is read.
struct EsdgTraces {
  const double* lo;
  const double* hi;
  int nv;
  int bgmode;
};

// the two directions other than d, in increasing order
__host__ __device__ inline void esdg_others(int d, int& o1, int& o2) {
  o1 = (d == 0) ? 1 : 0;
  o2 = (d == 2) ? 1 : 2;
}

__host__ __device__ inline int esdg_node(int Nq, int i, int j, int k) { return i + Nq * (j + Nq * k); }

// face id of plane P in direction d at transverse element indices (a, b)
__host__ __device__ inline long long esdg_face_id(const EsdgGrid& g, int d, int P, int a, int b) {
  int o1, o2;
  esdg_others(d, o1, o2);
  return g.face_off[d] + ((long long)P * g.K[o2] + b) * g.K[o1] + a;
}

#ifdef __CUDACC__
// Reciprocal in FP64 from the hardware approximation rcp.approx.ftz.f64
// (MUFU; relative error below 2^-19.9, measured on this GPU over 1M values)
// refined by one cubically convergent step: with e = 1 - x r0 the update
// r0 (1 + e + e^2) is the order-2 Householder step for f(r) = 1/r - x, leaving
// a truncation error e^3 < 2^-59, i.e. the result is within about one rounding
// of 1/x.  Three DFMA on the FP64 pipe; the seed runs on the MUFU pipe.
__device__ __forceinline__ double esdg_rcp(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  const double t = fma(e, e, e);
  return fma(r, t, r);
}

// Same seed with a single Newton step (relative error ~2^-39); used only where
// the result feeds a small correction term.
__device__ __forceinline__ double esdg_rcp_lo(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// IEEE-754 double <-> float repacking with integer instructions.  cvt.f32.f64
// and cvt.f64.f32 occupy the FP64 pipe on this GPU, which is the bottleneck of
// the FP64 kernels; these run on the integer pipes.
// esdg_d2f rounds to nearest even like cvt.rn.f32.f64 for every |x| < 2^128
// whose result is a normal float (a rounding past FLT_MAX gives the signed
// infinity); magnitudes below the float normal range flush to a signed zero.
// Larger magnitudes, infinities and NaNs are outside its domain (the value is
// unspecified): the kernels convert only state-derived values, which lie far
// inside the range unless the run has diverged, and a diverged state is
// reported by the stage update's status word (the FP64 state itself carries
// the non-finite values), so the hot paths spend no instructions on them.
// esdg_f2d is exact for normal floats, infinities and NaNs; zero and
// subnormal floats give +-0.  (Both are checked against the IEEE conversions
// by the numeric test hook.)
__device__ __forceinline__ float esdg_d2f(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned rest = lo & 0x1fffffffu;
  const unsigned sign = hi & 0x80000000u;
  unsigned f = sign | ((unsigned)e << 23) | m;
  f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (f & 1u));
  return (e <= 0) ? __uint_as_float(sign) : __uint_as_float(f);
}
__device__ __forceinline__ double esdg_f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  const unsigned eb = e == 0xffu ? 0x7ffu : e + 896u;  // infinities and NaNs keep all ones
  const unsigned hi = (u & 0x80000000u) | (eb << 20) | (m >> 3);
  return (e == 0) ? __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32))
                  : __longlong_as_double((long long)(((unsigned long long)hi << 32) | (m << 29)));
}
// x * 2^k (|k| small) with an integer add on the exponent field instead of an
// FP64-pipe multiply: exact for normal x and normal results; infinities and
// NaNs pass through; zero and subnormal inputs, and results below the normal
// range, give a signed zero (flush to zero); overflow gives a signed infinity.
// (Velocities in the far tail of a Gaussian perturbation do reach the
// subnormal range, so the guards are needed.)
__device__ __forceinline__ double esdg_ldexp(double x, int k) {
  const int hi = __double2hiint(x);
  const int ef = (hi >> 20) & 0x7ff, nf = ef + k;
  const int sign = hi & (int)0x80000000;
  if (ef == 0x7ff) return x;
  if (ef == 0 || nf <= 0) return __hiloint2double(sign, 0);
  if (nf >= 0x7ff) return __hiloint2double(sign | 0x7ff00000, 0);
  return __hiloint2double(hi + k * (1 << 20), __double2loint(x));
}

// ---- 1-D bulk copies (the TMA engine) completing on a shared-memory mbarrier
__device__ __forceinline__ unsigned esdg_smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void esdg_mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(esdg_smem_addr(bar)), "r"(count)
               : "memory");
}
// make barrier initialisation visible to the async proxy (the copy engine)
__device__ __forceinline__ void esdg_fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this CTA's earlier generic shared-memory accesses before later async-proxy writes
__device__ __forceinline__ void esdg_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void esdg_mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(esdg_smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared, 16-byte aligned addresses, bytes a multiple of 16
__device__ __forceinline__ void esdg_bulk_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          esdg_smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(esdg_smem_addr(bar))
      : "memory");
}
// Wait for completion of the barrier phase with the given parity, at most
// `limit` polls (each poll may suspend the thread briefly); false if the limit
// ran out.
__device__ __forceinline__ bool esdg_mbar_wait(unsigned long long* bar, unsigned parity,
                                               unsigned limit) {
  const unsigned a = esdg_smem_addr(bar);
  for (unsigned it = 0; it < limit; it++) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// The shift of a block's data in its shared-memory copy target: the bulk copy
// starts at the 16-byte boundary at or below src, so the block's first element
// lands (src mod 16) / sizeof(T) elements into the target.
template <typename T>
__device__ __forceinline__ int esdg_block_shift(const T* src) {
  constexpr unsigned long long K = 16 / sizeof(T);
  return (int)((reinterpret_cast<unsigned long long>(src) / sizeof(T)) % K);
}
template <typename T>
__device__ __forceinline__ void esdg_cp_async(T* dst, const T* src) {  // sizeof(T) bytes
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(esdg_smem_addr(dst)), "l"(src),
               "n"((int)sizeof(T))
               : "memory");
}
__device__ __forceinline__ void esdg_cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// A state value the stage update must flag: an infinity or a NaN (exponent
// field all ones), or, for a density (dens = true), a value that is not
// positive.  Integer tests only.
__device__ __forceinline__ bool esdg_bad_state(double x, bool dens) {
  const long long b = __double_as_longlong(x);
  return ((int)(b >> 32) & 0x7ff00000) == 0x7ff00000 || (dens && b <= 0);
}
// x < y for non-negative doubles, compared as integers (no FP64-pipe compare)
__device__ __forceinline__ bool esdg_lt_pos(double x, double y) {
  return __double_as_longlong(x) < __double_as_longlong(y);
}

__device__ __forceinline__ float esdg_rcpf(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Log-mean series.  With f = (a - b)/(a + b), u = f^2:
//   ln(a/b) = 2 f A(u),  A(u) = sum_k u^k / (2k + 1),
//   <a>_log = (a - b)/ln(a/b) = {{a}} Q(u),  Q = 1/A = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
// (coefficients of f/artanh f).  For u < 1e-4 four terms leave a truncation
// error below 2e-17.
#define ESDG_LOG_EPS 1.0e-4
// FP64 series with the tail in FP32: for u < 1e-4 the terms beyond u^1 are below
// 2e-9 in size, so evaluating them in FP32 (relative error ~2^-22) perturbs the
// result by < 1e-16 of its value; two DFMA instead of three.  Used on the
// series path of the FP64 volume kernel, where every pair has u < 1e-4.  The
// conversions are short integer sequences (they sit on the pair's dependency
// chain): u -> float by truncating the mantissa, the positive tail back by
// re-biasing the exponent.
__device__ __forceinline__ float esdg_d2f_tail(double u) {  // 0 <= u < 2^128
  const int hi = __double2hiint(u);
  const unsigned lo = (unsigned)__double2loint(u);
  const float f = __uint_as_float(__funnelshift_l(lo, (unsigned)(hi - 0x38000000), 3));
  return hi < 0x38100000 ? 0.0f : f;  // below the float normal range: 0
}
__device__ __forceinline__ double esdg_f2d_pos(float f) {  // positive normal f
  const unsigned b = __float_as_uint(f);
  return __hiloint2double((int)((b >> 3) + 0x38000000u), (int)(b << 29));
}
__device__ __forceinline__ double esdg_A_t(double u) {
  const float tail = fmaf(esdg_d2f_tail(u), 1.0f / 7.0f, 1.0f / 5.0f);
  return fma(u, fma(u, esdg_f2d_pos(tail), 1.0 / 3.0), 1.0);
}
__device__ __forceinline__ double esdg_Q2_t(double u) {
  const float tail = fmaf(esdg_d2f_tail(u), 88.0f / 945.0f, 8.0f / 45.0f);  // -(u^2 coefficient tail)
  return fma(-u, fma(u, esdg_f2d_pos(tail), 2.0 / 3.0), 2.0);
}
// FP32 variants: for u < 2e-2 the four-term truncation error is below 2e-8.
#define ESDG_LOG_EPS32 2.0e-2f
__device__ __forceinline__ float esdg_Af(float u) {
  return fmaf(u, fmaf(u, fmaf(u, 1.0f / 7.0f, 1.0f / 5.0f), 1.0f / 3.0f), 1.0f);
}
__device__ __forceinline__ float esdg_Qf(float u) {
  return fmaf(u, fmaf(u, fmaf(u, -44.0f / 945.0f, -4.0f / 45.0f), -1.0f / 3.0f), 1.0f);
}
__device__ __forceinline__ float esdg_Q2f(float u) {
  return fmaf(u, fmaf(u, fmaf(u, -88.0f / 945.0f, -8.0f / 45.0f), -2.0f / 3.0f), 2.0f);
}

#endif  // __CUDACC__

// ---- launch wrappers implemented in the kernel translation units ----------
cudaError_t esdg_launch_geometry(const EsdgGrid& g, const EsdgLGL& L, double* x, double* J,
                                 double* Ja, double* vgeo, float* vgeo32, double* fgeo,
                                 const EsdgPhys& P, cudaStream_t s);
cudaError_t esdg_launch_bubble(const EsdgGrid& g, const EsdgPhys& P, const double* x, double theta0,
                               double amp, const double* centre, double radius, int sharp,
                               double* q, cudaStream_t s);
// amp: amplitude of the Gaussian wind perturbation (m/s); 0 gives the balanced jet alone
cudaError_t esdg_launch_channel(const EsdgGrid& g, const EsdgPhys& P, const double* x, double* q,
                                double amp, cudaStream_t s);
cudaError_t esdg_launch_background(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                   const double* q, double* bg, double* q0, cudaStream_t s);
// bgq: a moving background's state [E][5][np] (mixed with bg only; null at rest).
// Faces f0 .. f1 - 1 only (global face ids; f1 < 0: to the last face).
cudaError_t esdg_launch_face(const EsdgGrid& g, const EsdgPhys& P, int mixed, const double* q,
                             const double* fgeo, void* fflux, cudaStream_t s,
                             const double* bg = nullptr,
                             EsdgTraces tr = EsdgTraces{nullptr, nullptr, 5, 0},
                             const double* bgq = nullptr, long long f0 = 0, long long f1 = -1);
// Pack a partition's own traces for its neighbours: the state of the first
// element layer's i = 0 nodes into send_lo (if remote[0]) and of the last
// layer's i = N nodes into send_hi (if remote[1]), layout of EsdgTraces.
cudaError_t esdg_launch_trace_pack(const EsdgGrid& g, const double* q, const double* bg, int nv,
                                   double* send_lo, double* send_hi, cudaStream_t s);
// The mixed volume kernels' background copy (bg3: rho_bg, E_bg, phi FP64; bgp:
// rho_bg/4, b_bg/2, 1/b_bg, p_bg FP32) from the stored background bg.
cudaError_t esdg_launch_background_vol(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                       const double* bg, double* bg3, float* bgp, cudaStream_t s);
// A moving background's FP32 velocity u_bg = m_bg/rho_bg from its state bgq
// ([E][5][np]) into bgu ([E][3][np]).
cudaError_t esdg_launch_background_velocity(const EsdgGrid& g, const double* bgq, float* bgu,
                                            cudaStream_t s);
// dst[i] = src[i] rounded to FP32, i < n
cudaError_t esdg_launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s);
// The background state at rest from the stored background, per node:
// (rho_bg, 0, 0, 0, p_bg/(gamma-1) + rho_bg phi) -- the expression the
// background kernel uses, so the result equals its own at-rest state.
cudaError_t esdg_launch_background_state(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                         const double* bg, double* q0, cudaStream_t s);
// mode 0: write rhs; mode 1: fused LSRK stage (dq, q updated in place)
struct EsdgVolArgs {
  const double* q_in;    // state read by the prologue and the source term
  double* q_io;          // mode 1: state updated in place (may equal q_in)
  void* dq;              // mode 1: RK register (double in FP64 mode, float in mixed mode)
  double* rhs;           // mode 0: right-hand side output
  const void* vgeo;      // [E][11][np] double (FP64) or float (mixed)
  const double* vgeo64;  // [E][11][np] double (geopotential for the pressure recovery)
  const void* fflux;     // face fluxes, double or float
  const double* x;       // coordinates (Coriolis parameter)
  const double* bg;      // mixed mode with a background: [E][3][np] rho_bg, E_bg, phi (else null)
  const float* bgp;      // mixed mode with a background: [E][4][np] rho_bg/4, b_bg/2, 1/b_bg, p_bg
  const float* rhs_bg;   // mixed mode with a background: [E][3][np] momentum rhs of it (FP32)
  // a moving background (one that carries a flow, e.g. a balanced jet); null at rest:
  const double* bgq;     // [E][5][np] the background state itself (rho_bg, m_bg, E_bg)
  const float* bgu;      // [E][3][np] u_bg in FP32
  const float* rhs_bgm;  // [E][5][np] the background's full right-hand side (FP32)
  double rkA, rkB, dt;
  int* status;           // mode 1: set to 1 when an updated state value is not finite or a
                         // density is not positive (null: not checked)
};
// The mixed volume kernel with a moving background (per-tile kernel; its own
// translation unit): mode 0 writes rhs, mode 1 applies the LSRK stage.
cudaError_t esdg_launch_volume_mixed_moving(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                            int mode, const EsdgVolArgs& a, cudaStream_t s);
// One mesh of a batch: everything its kernels need, read by the persistent
// batched kernels from a device array (one entry per resident solve).
struct EsdgMember {
  EsdgGrid g;
  EsdgPhys P;
  EsdgVolArgs a;       // q_in == q_io: the member's state; dq, geometry, face fluxes, dt
  const double* fgeo;  // face geometry
  const double* bg;    // mixed background (rho_bg, b_bg, p_bg, for the faces) or null
  // (sizeof a multiple of 16 bytes: the pipelined kernels bulk-copy descriptors)
};

// Batched persistent launches over device work tables (tiles: int2 (member,
// first element) for the volume, (member, first face node) in blocks of 256
// for the faces; ntiles in device memory so the tables can change under a
// captured graph).  variant selects the tile shape (elements per CTA).
cudaError_t esdg_launch_face_batch(int N, int mixed, int bg, const EsdgMember* members,
                                   const int2* tiles, const int* ntiles, int grid, cudaStream_t s);
// what: 0 launch (returns 0 or -1), 1 elements per tile, 2 CTAs per SM
int esdg_volume_batch_f64(int what, int N, int variant, const EsdgMember* members, const int2* tiles,
                          const int* ntiles, int grid, const EsdgLGL& L, double A, double B,
                          cudaStream_t s);
int esdg_volume_batch_mixed(int what, int N, int variant, const EsdgMember* members,
                            const int2* tiles, const int* ntiles, int grid, const EsdgLGL& L,
                            double A, double B, cudaStream_t s);
int esdg_volume_batch_variants_f64(int N);
int esdg_volume_batch_variants_mixed(int N);

// Test hook (es_dg_debug_inject_wait_timeout): bytes the next single-mesh
// pipelined volume launch registers on its first barrier without copying them;
// read and cleared by the launcher.
unsigned esdg_take_phantom();
// 1 if a bounded wait of the pipelined FP64 / mixed volume kernels ran out
// since the last call (the flag is cleared), 0 if not, -1 on a CUDA error
int esdg_volume_f64_take_timeout();
int esdg_volume_mixed_take_timeout();
cudaError_t esdg_launch_volume_f64(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, int mode,
                                   const EsdgVolArgs& a, cudaStream_t s);
cudaError_t esdg_launch_volume_mixed(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                     int mode, const EsdgVolArgs& a, cudaStream_t s);
#ifdef __CUDACC__
inline cudaError_t esdg_launch_volume(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                      int mixed, int mode, const EsdgVolArgs& a, cudaStream_t s) {
  return mixed ? esdg_launch_volume_mixed(g, L, P, mode, a, s)
               : esdg_launch_volume_f64(g, L, P, mode, a, s);
}
#endif
// Reductions with a scratch buffer of at least esdg_reduce_scratch(g) doubles;
// the result lands in out[0] (CFL: 1 / the largest reference-space signal
// speed) or out[0..2] (integrals: mass, energy, entropy), device memory.
size_t esdg_reduce_scratch(const EsdgGrid& g);
cudaError_t esdg_launch_cfl(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, const double* q,
                            const double* x, const double* J, const double* Ja, double* scratch,
                            double* out, cudaStream_t s);
cudaError_t esdg_launch_integrals(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                  const double* q, const double* J, const double* x,
                                  double* scratch, double* out, cudaStream_t s);
int esdg_lgl_build(int N, EsdgLGL* out);
