// surface.cu -- interface and wall flux (Section 3: the surface term of
// Eq. (nm:semi) with the entropy-conservative flux plus matrix dissipation).
//
// One thread per face node.  For face (d, P) the "-" state is the element
// below the plane and the "+" state the element above it; at a wall the missing
// side is the mirror state (rho, U - 2 (U . nhat) nhat, E).  The kernel writes
// (s / w_end) F*(q-, q+, nhat) with nhat along +d; the volume kernel lifts it
// into both elements with opposite signs, so every face is evaluated once.
//
// Interface flux: F* = F#(q-, q+; nhat) - 1/2 R |Lambda| T R^T [[v]] with the
// averaged state rho_hat = <rho>_log, u = {{u}}, p_hat = {{rho}}/(2{{b}}),
// a^2 = gamma p_hat/rho_hat, H = a^2/(gamma-1) + |u|^2/2 + phi.  The shear
// part is applied without tangent vectors: p_hat |u_n| (0, y_t, u . y_t),
// y_t = (I - nhat nhat^T)([[v]]_m + u [[v]]_E).  Jumps of log rho and log b come
// from the same artanh series as the log means; log p = log rho - log b - log 2.
#include "esdg_internal.cuh"

namespace {

template <typename R>
struct FaceMath;

template <>
struct FaceMath<double> {
  static __device__ __forceinline__ double rcp(double x) { return esdg_rcp(x); }
  static __device__ __forceinline__ double A(double u) { return esdg_A(u); }
  static __device__ __forceinline__ double Q(double u) { return esdg_Q(u); }
  static __device__ __forceinline__ bool small(double u) { return (float)u < (float)ESDG_LOG_EPS; }
  // ln(p/m) by per-side logarithms (the log branch of the log mean)
  static __device__ __forceinline__ double ljump(double p, double m, double diff) {
    return log(p) - log(m);
  }
  static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
};

template <>
struct FaceMath<float> {
  static __device__ __forceinline__ float rcp(float x) { return esdg_rcpf(x); }
  static __device__ __forceinline__ float A(float u) { return esdg_Af(u); }
  static __device__ __forceinline__ float Q(float u) { return esdg_Qf(u); }
  static __device__ __forceinline__ bool small(float u) { return u < ESDG_LOG_EPS32; }
  // ln(p/m) = log1p((p - m)/m): no cancellation between two large logarithms
  static __device__ __forceinline__ float ljump(float p, float m, float diff) {
    return log1pf(diff * esdg_rcpf(m));
  }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
};

template <typename R>
struct Side {
  R rho, u0, u1, u2, b;
};

// primitives from the FP64 state: the pressure (and with it b = rho/(2p)) is
// always recovered in FP64, where E - rho phi cancels
template <typename R>
__device__ __forceinline__ Side<R> side_from(const double* q, double phi, double gm1) {
  const double rho = q[0];
  const double ir = esdg_rcp(rho);
  const double u0 = q[1] * ir, u1 = q[2] * ir, u2 = q[3] * ir;
  double e = fma(-rho, phi, q[4]);
  e = fma(-0.5 * q[1], u0, e);
  e = fma(-0.5 * q[2], u1, e);
  e = fma(-0.5 * q[3], u2, e);
  const double p = gm1 * e;
  Side<R> s;
  s.rho = (R)rho;
  s.u0 = (R)u0;
  s.u1 = (R)u1;
  s.u2 = (R)u2;
  s.b = (R)(0.5 * rho * esdg_rcp(p));
  return s;
}

template <typename R>
__device__ __forceinline__ void face_flux(const Side<R>& M, const Side<R>& Pp, R phi, R n0, R n1,
                                          R n2, R gamma, int dissipation, R* F) {
  using Mth = FaceMath<R>;
  const R gm1 = gamma - (R)1;
  const R half = (R)0.5;
  // log means and log jumps of rho and b
  const R sr = Pp.rho + M.rho, dr = Pp.rho - M.rho;
  const R sb = Pp.b + M.b, db = Pp.b - M.b;
  const R rsr = Mth::rcp(sr), rsb = Mth::rcp(sb);
  const R fr = dr * rsr, ur = fr * fr;
  const R fb = db * rsb, ub = fb * fb;
  R rho_log, lnr_jump, iblog, lnb_jump;
  if (Mth::small(ur)) {
    const R Ar = Mth::A(ur);
    rho_log = half * sr * Mth::Q(ur);
    lnr_jump = (R)2 * fr * Ar;
  } else {
    lnr_jump = Mth::ljump(Pp.rho, M.rho, dr);
    rho_log = dr / lnr_jump;
  }
  if (Mth::small(ub)) {
    const R Ab = Mth::A(ub);
    iblog = (R)2 * rsb * Ab;
    lnb_jump = (R)2 * fb * Ab;
  } else {
    lnb_jump = Mth::ljump(Pp.b, M.b, db);
    iblog = lnb_jump / db;
  }
  const R u0 = half * (M.u0 + Pp.u0), u1 = half * (M.u1 + Pp.u1), u2 = half * (M.u2 + Pp.u2);
  const R un = u0 * n0 + u1 * n1 + u2 * n2;
  const R pt = sr * rsb * half;  // {{rho}} / (2 {{b}})
  const R uu = M.u0 * Pp.u0 + M.u1 * Pp.u1 + M.u2 * Pp.u2;
  const R Fr = rho_log * un;
  F[0] = Fr;
  F[1] = Fr * u0 + pt * n0;
  F[2] = Fr * u1 + pt * n1;
  F[3] = Fr * u2 + pt * n2;
  F[4] = Fr * (iblog / ((R)2 * gm1) + half * uu + phi) + pt * un;
  if (!dissipation) return;
  // entropy-variable jumps
  const R bu2m = M.b * (M.u0 * M.u0 + M.u1 * M.u1 + M.u2 * M.u2);
  const R bu2p = Pp.b * (Pp.u0 * Pp.u0 + Pp.u1 * Pp.u1 + Pp.u2 * Pp.u2);
  const R jv1 = lnr_jump + lnb_jump / gm1 - (bu2p - bu2m) + (R)2 * phi * db;
  const R jm0 = (R)2 * (Pp.b * Pp.u0 - M.b * M.u0);
  const R jm1 = (R)2 * (Pp.b * Pp.u1 - M.b * M.u1);
  const R jm2 = (R)2 * (Pp.b * Pp.u2 - M.b * M.u2);
  const R jv5 = (R)-2 * db;
  // averaged state and wave strengths
  const R irho_hat = (R)2 * rsr * Mth::A(ur);  // 1/<rho>_log (series branch)
  const R irh = Mth::small(ur) ? irho_hat : lnr_jump / dr;
  const R a2 = gamma * pt * irh;
  const R a = Mth::sq(a2);
  const R k2 = half * (u0 * u0 + u1 * u1 + u2 * u2) + phi;
  const R H = a2 / gm1 + k2;
  const R njm = n0 * jm0 + n1 * jm1 + n2 * jm2;
  const R w2 = jv1 + u0 * jm0 + u1 * jm1 + u2 * jm2 + k2 * jv5;
  const R ac = a2 / gm1 * jv5;
  const R w1 = w2 - a * njm + ac - a * un * jv5;
  const R w5 = w2 + a * njm + ac + a * un * jv5;
  const R ig = (R)1 / gamma;
  const R c1 = fabs(un - a) * rho_log * half * ig * w1;
  const R c2 = fabs(un) * rho_log * gm1 * ig * w2;
  const R c5 = fabs(un + a) * rho_log * half * ig * w5;
  const R ls = fabs(un) * pt;
  // shear part, tangent-free
  const R y0 = jm0 + u0 * jv5, y1 = jm1 + u1 * jv5, y2 = jm2 + u2 * jv5;
  const R yn = y0 * n0 + y1 * n1 + y2 * n2;
  const R t0 = y0 - yn * n0, t1 = y1 - yn * n1, t2 = y2 - yn * n2;
  const R csum = c1 + c2 + c5, cdif = c5 - c1;
  const R d0 = csum;
  const R dm0 = csum * u0 + a * cdif * n0 + ls * t0;
  const R dm1 = csum * u1 + a * cdif * n1 + ls * t1;
  const R dm2 = csum * u2 + a * cdif * n2 + ls * t2;
  const R dE = (c1 + c5) * H + a * un * cdif + c2 * k2 + ls * (u0 * t0 + u1 * t1 + u2 * t2);
  F[0] -= half * d0;
  F[1] -= half * dm0;
  F[2] -= half * dm1;
  F[3] -= half * dm2;
  F[4] -= half * dE;
}

template <typename R, int N>
__global__ void __launch_bounds__(256) k_face(EsdgGrid g, EsdgPhys P, const double* __restrict__ q,
                                              const double* __restrict__ fgeo,
                                              R* __restrict__ fflux) {
  constexpr int Nq = N + 1, NF2 = Nq * Nq, NP = Nq * Nq * Nq;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.nfaces * NF2) return;
  const long long f = tid / NF2;
  const int fn = (int)(tid - f * NF2);
  int d = 0;
  while (d < 2 && f >= g.face_off[d + 1]) d++;
  int o1, o2;
  esdg_others(d, o1, o2);
  long long r = f - g.face_off[d];
  const int a = (int)(r % g.K[o1]);
  r /= g.K[o1];
  const int b = (int)(r % g.K[o2]);
  const int Pl = (int)(r / g.K[o2]);
  const int Kd = g.K[d];
  // elements below and above the plane (-1 at a wall)
  int em = -1, ep = -1;
  {
    int idx[3];
    idx[o1] = a;
    idx[o2] = b;
    if (Pl > 0 || g.periodic[d]) {
      idx[d] = (Pl - 1 + Kd) % Kd;
      em = idx[0] + g.K[0] * (idx[1] + g.K[1] * idx[2]);
    }
    if (Pl < Kd) {
      idx[d] = Pl;
      ep = idx[0] + g.K[0] * (idx[1] + g.K[1] * idx[2]);
    }
  }
  int ijk[3];
  ijk[o1] = fn % Nq;
  ijk[o2] = fn / Nq;
  ijk[d] = N;
  const int nm = esdg_node(Nq, ijk[0], ijk[1], ijk[2]);
  ijk[d] = 0;
  const int npn = esdg_node(Nq, ijk[0], ijk[1], ijk[2]);
  const double* G = fgeo + (size_t)f * 5 * NF2;
  const double n0 = G[0 * NF2 + fn], n1 = G[1 * NF2 + fn], n2 = G[2 * NF2 + fn];
  const double scale = G[3 * NF2 + fn], phi = G[4 * NF2 + fn];
  double qm[5], qp[5];
  if (em >= 0)
    for (int v = 0; v < 5; v++) qm[v] = q[((size_t)em * 5 + v) * NP + nm];
  if (ep >= 0)
    for (int v = 0; v < 5; v++) qp[v] = q[((size_t)ep * 5 + v) * NP + npn];
  if (em < 0 || ep < 0) {  // reflecting wall: mirror the existing side
    const double* src = (em < 0) ? qp : qm;
    double* dst = (em < 0) ? qm : qp;
    const double Un = src[1] * n0 + src[2] * n1 + src[3] * n2;
    dst[0] = src[0];
    dst[1] = src[1] - 2.0 * Un * n0;
    dst[2] = src[2] - 2.0 * Un * n1;
    dst[3] = src[3] - 2.0 * Un * n2;
    dst[4] = src[4];
  }
  const double gm1 = P.gamma - 1.0;
  const Side<R> M = side_from<R>(qm, phi, gm1), Pp = side_from<R>(qp, phi, gm1);
  R F[5];
  face_flux<R>(M, Pp, (R)phi, (R)n0, (R)n1, (R)n2, (R)P.gamma, P.dissipation, F);
  R* out = fflux + (size_t)f * 5 * NF2;
  const R sc = (R)scale;
#pragma unroll
  for (int v = 0; v < 5; v++) out[v * NF2 + fn] = sc * F[v];
}

template <typename R>
cudaError_t launch_face_t(const EsdgGrid& g, const EsdgPhys& P, const double* q, const double* fgeo,
                          R* fflux, cudaStream_t s) {
  const long long nt = g.nfaces * g.Nq * g.Nq;
  if (nt == 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nt + 255) / 256);
  switch (g.N) {
    case 1: k_face<R, 1><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 2: k_face<R, 2><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 3: k_face<R, 3><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 4: k_face<R, 4><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 5: k_face<R, 5><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 6: k_face<R, 6><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    case 7: k_face<R, 7><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t esdg_launch_face(const EsdgGrid& g, const EsdgPhys& P, int mixed, const double* q,
                             const double* fgeo, void* fflux, cudaStream_t s) {
  if (mixed) return launch_face_t<float>(g, P, q, fgeo, (float*)fflux, s);
  return launch_face_t<double>(g, P, q, fgeo, (double*)fflux, s);
}
