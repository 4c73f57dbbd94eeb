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
  // 2 A(u) and Q(u)/2 with the tails beyond u^1 in FP32 (u < 1e-4: the tails are
  // below 4e-9, their FP32 rounding below 1e-16 of the result)
  static __device__ __forceinline__ double A2(double u) {
    const float tail = fmaf(esdg_d2f_tail(u), 2.0f / 7.0f, 2.0f / 5.0f);
    return fma(u, fma(u, esdg_f2d_pos(tail), 2.0 / 3.0), 2.0);
  }
  static __device__ __forceinline__ double Qh(double u) {
    const float tail = fmaf(esdg_d2f_tail(u), 22.0f / 945.0f, 2.0f / 45.0f);
    return fma(-u, fma(u, esdg_f2d_pos(tail), 1.0 / 6.0), 0.5);
  }
  static __device__ __forceinline__ bool small(double u) { return esdg_lt_pos(u, ESDG_LOG_EPS); }
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
  static __device__ __forceinline__ float A2(float u) { return 2.0f * esdg_Af(u); }
  static __device__ __forceinline__ float Qh(float u) { return 0.5f * esdg_Qf(u); }
  static __device__ __forceinline__ bool small(float u) { return u < ESDG_LOG_EPS32; }
  // ln(p/m) = log1p((p - m)/m): no cancellation between two large logarithms
  static __device__ __forceinline__ float ljump(float p, float m, float diff) {
    return log1pf(diff * esdg_rcpf(m));
  }
  static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
};

// double -> R without the FP64-pipe conversion instruction
template <typename R>
__device__ __forceinline__ R to_r(double x) {
  if constexpr (sizeof(R) == sizeof(float)) return esdg_d2f(x);
  else return x;
}

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
  // halvings on the exponent field (esdg_ldexp): no FP64-pipe instruction
  double e = fma(-rho, phi, q[4]);
  e = fma(-esdg_ldexp(q[1], -1), u0, e);
  e = fma(-esdg_ldexp(q[2], -1), u1, e);
  e = fma(-esdg_ldexp(q[3], -1), u2, e);
  const double p = gm1 * e;
  const double b = esdg_ldexp(rho, -1) * esdg_rcp(p);  // rho/(2p)
  Side<R> s;
  if constexpr (sizeof(R) == sizeof(float)) {
    s.rho = esdg_d2f(rho);
    s.u0 = esdg_d2f(u0);
    s.u1 = esdg_d2f(u1);
    s.u2 = esdg_d2f(u2);
    s.b = esdg_d2f(b);
  } else {
    s.rho = rho;
    s.u0 = u0;
    s.u1 = u1;
    s.u2 = u2;
    s.b = b;
  }
  return s;
}

// x * 2 and x / 2 on the exponent field for doubles (no FP64-pipe instruction;
// esdg_ldexp: exact for normal values, subnormals flushed to zero)
template <typename R>
__device__ __forceinline__ R twice(R x) {
  if constexpr (sizeof(R) == sizeof(double)) return esdg_ldexp(x, 1);
  else return 2.0f * x;
}
template <typename R>
__device__ __forceinline__ R halfof(R x) {
  if constexpr (sizeof(R) == sizeof(double)) return esdg_ldexp(x, -1);
  else return 0.5f * x;
}

template <typename R>
__device__ __forceinline__ void face_flux(const Side<R>& M, const Side<R>& Pp, R phi, R n0, R n1,
                                          R n2, R gamma, R igm1, R igamma, int dissipation, R* F) {
  using Mth = FaceMath<R>;
  const R gm1 = gamma - (R)1;
  // log means and log jumps of rho and b
  const R sr = Pp.rho + M.rho, dr = Pp.rho - M.rho;
  const R sb = Pp.b + M.b, db = Pp.b - M.b;
  const R rsr = Mth::rcp(sr), rsb = Mth::rcp(sb);
  const R fr = dr * rsr, ur = fr * fr;
  const R fb = db * rsb, ub = fb * fb;
  R rho_log, lnr_jump, iblog, lnb_jump;
  const bool sr_small = Mth::small(ur);
  const R A2r = Mth::A2(ur);  // 2 A(u_rho), also 1/<rho>_log below
  if (sr_small) {
    rho_log = sr * Mth::Qh(ur);
    lnr_jump = fr * A2r;
  } else {
    lnr_jump = Mth::ljump(Pp.rho, M.rho, dr);
    rho_log = dr / lnr_jump;
  }
  if (Mth::small(ub)) {
    const R A2b = Mth::A2(ub);
    iblog = rsb * A2b;
    lnb_jump = fb * A2b;
  } else {
    lnb_jump = Mth::ljump(Pp.b, M.b, db);
    iblog = lnb_jump / db;
  }
  const R u0 = halfof(M.u0 + Pp.u0), u1 = halfof(M.u1 + Pp.u1), u2 = halfof(M.u2 + Pp.u2);
  const R un = fma(u2, n2, fma(u1, n1, u0 * n0));
  const R pt = halfof(sr * rsb);  // {{rho}} / (2 {{b}})
  const R uu = fma(M.u2, Pp.u2, fma(M.u1, Pp.u1, M.u0 * Pp.u0));
  const R Fr = rho_log * un;
  F[0] = Fr;
  F[1] = fma(Fr, u0, pt * n0);
  F[2] = fma(Fr, u1, pt * n1);
  F[3] = fma(Fr, u2, pt * n2);
  // F^E = F^rho (1/(2 (gamma-1) <b>_log) + u-.u+/2 + phi) + p* u_n
  F[4] = fma(Fr, fma(iblog, halfof(igm1), fma((R)0.5, uu, phi)), pt * un);
  if (!dissipation) return;
  // entropy-variable jumps
  const R bu2m = M.b * fma(M.u2, M.u2, fma(M.u1, M.u1, M.u0 * M.u0));
  const R bu2p = Pp.b * fma(Pp.u2, Pp.u2, fma(Pp.u1, Pp.u1, Pp.u0 * Pp.u0));
  const R jv1 = fma(twice(phi), db, fma(lnb_jump, igm1, lnr_jump) - (bu2p - bu2m));
  const R jm0 = twice(fma(Pp.b, Pp.u0, -M.b * M.u0));
  const R jm1 = twice(fma(Pp.b, Pp.u1, -M.b * M.u1));
  const R jm2 = twice(fma(Pp.b, Pp.u2, -M.b * M.u2));
  const R jv5 = -twice(db);
  // averaged state and wave strengths
  const R irh = sr_small ? rsr * A2r : lnr_jump / dr;  // 1/<rho>_log
  const R a2 = gamma * pt * irh;
  const R a = Mth::sq(a2);
  const R k2 = fma((R)0.5, fma(u2, u2, fma(u1, u1, u0 * u0)), phi);
  const R a2g = a2 * igm1;
  const R H = a2g + k2;
  const R njm = fma(n2, jm2, fma(n1, jm1, n0 * jm0));
  const R w2 = fma(k2, jv5, fma(u2, jm2, fma(u1, jm1, fma(u0, jm0, jv1))));
  const R aun = a * un, anjm = a * njm;
  const R w2a = fma(a2g, jv5, w2);
  const R w1 = fma(-aun, jv5, w2a - anjm);
  const R w5 = fma(aun, jv5, w2a + anjm);
  const R rlh = rho_log * halfof(igamma), rlg = rho_log * (gm1 * igamma);
  const R c1 = fabs(un - a) * rlh * w1;
  const R c2 = fabs(un) * rlg * w2;
  const R c5 = fabs(un + a) * rlh * w5;
  const R ls = fabs(un) * pt;
  // shear part, tangent-free
  const R y0 = fma(u0, jv5, jm0), y1 = fma(u1, jv5, jm1), y2 = fma(u2, jv5, jm2);
  const R yn = fma(y2, n2, fma(y1, n1, y0 * n0));
  const R t0 = fma(-yn, n0, y0), t1 = fma(-yn, n1, y1), t2 = fma(-yn, n2, y2);
  const R csum = c1 + c2 + c5, cdif = c5 - c1;
  const R acd = a * cdif;
  const R dm0 = fma(csum, u0, fma(acd, n0, ls * t0));
  const R dm1 = fma(csum, u1, fma(acd, n1, ls * t1));
  const R dm2 = fma(csum, u2, fma(acd, n2, ls * t2));
  const R ut = fma(u2, t2, fma(u1, t1, u0 * t0));
  const R dE = fma(c1 + c5, H, fma(aun, cdif, fma(c2, k2, ls * ut)));
  F[0] = fma((R)-0.5, csum, F[0]);
  F[1] = fma((R)-0.5, dm0, F[1]);
  F[2] = fma((R)-0.5, dm1, F[2]);
  F[3] = fma((R)-0.5, dm2, F[3]);
  F[4] = fma((R)-0.5, dE, F[4]);
}

// Jumps and pressure mean of a face node relative to a background, formed from
// FP64 differences (see face_node): [[rho]], [[b]], [[b u]], [[b |u|^2]] and
// p* - p_bg, each with its FP32 rounding relative to the perturbations and jumps.
struct BgFace {
  float dr, db, dbu0, dbu1, dbu2, dbuu, ptp;
};

// The matrix dissipation of the face flux from the jumps J (FP32, relative to
// the perturbations) and the averaged state: F -= 1/2 R |Lambda| T R^T [[v]].
__device__ __forceinline__ void dissipate_bg(float phi, float n0, float n1, float n2, float gamma,
                                             float igm1, float igamma, const BgFace& J,
                                             bool r_small, float rsr, float ur, float lnr_jump,
                                             float lnb_jump, float rho_log, float pt, float u0,
                                             float u1, float u2, float un, float* F) {
  using Mth = FaceMath<float>;
  const float gm1 = gamma - 1.0f;
  const float half = 0.5f;
  const float dr = J.dr, db = J.db;
  const float jv1 = lnr_jump + lnb_jump * igm1 - J.dbuu + 2.0f * phi * db;
  const float jm0 = 2.0f * J.dbu0, jm1 = 2.0f * J.dbu1, jm2 = 2.0f * J.dbu2;
  const float jv5 = -2.0f * db;
  const float irh = r_small ? 2.0f * rsr * Mth::A(ur) : lnr_jump / dr;
  const float a2 = gamma * pt * irh;
  const float a = sqrtf(a2);
  const float k2 = half * (u0 * u0 + u1 * u1 + u2 * u2) + phi;
  const float a2g = a2 * igm1;
  const float H = a2g + k2;
  const float njm = n0 * jm0 + n1 * jm1 + n2 * jm2;
  const float w2 = jv1 + u0 * jm0 + u1 * jm1 + u2 * jm2 + k2 * jv5;
  const float ac = a2g * jv5;
  const float w1 = w2 - a * njm + ac - a * un * jv5;
  const float w5 = w2 + a * njm + ac + a * un * jv5;
  const float c1 = fabsf(un - a) * rho_log * half * igamma * w1;
  const float c2 = fabsf(un) * rho_log * gm1 * igamma * w2;
  const float c5 = fabsf(un + a) * rho_log * half * igamma * w5;
  const float ls = fabsf(un) * pt;
  const float y0 = jm0 + u0 * jv5, y1 = jm1 + u1 * jv5, y2 = jm2 + u2 * jv5;
  const float yn = y0 * n0 + y1 * n1 + y2 * n2;
  const float t0 = y0 - yn * n0, t1 = y1 - yn * n1, t2 = y2 - yn * n2;
  const float csum = c1 + c2 + c5, cdif = c5 - c1;
  F[0] -= half * csum;
  F[1] -= half * (csum * u0 + a * cdif * n0 + ls * t0);
  F[2] -= half * (csum * u1 + a * cdif * n1 + ls * t1);
  F[3] -= half * (csum * u2 + a * cdif * n2 + ls * t2);
  F[4] -= half * ((c1 + c5) * H + a * un * cdif + c2 * k2 + ls * (u0 * t0 + u1 * t1 + u2 * t2));
}

// Mixed precision relative to a hydrostatic background (u_bg = 0, continuous
// across faces): the face flux's background part is the Euler flux
// (0, p_bg nhat, 0), so the kernel stores F* - (0, p_bg nhat, 0).  Its momentum
// pressure p* - p_bg and the jumps feeding the dissipation come in from BgFace,
// so FP32 rounding is relative to the perturbations and jumps, not to the state.
__device__ __forceinline__ void face_flux_bg(const Side<float>& M, const Side<float>& Pp, float phi,
                                             float n0, float n1, float n2, float gamma, float igm1,
                                             float igamma, int dissipation, const BgFace& J,
                                             float* F) {
  using Mth = FaceMath<float>;
  const float half = 0.5f;
  const float sr = Pp.rho + M.rho, dr = J.dr;
  const float sb = Pp.b + M.b, db = J.db;
  const float rsr = Mth::rcp(sr), rsb = Mth::rcp(sb);
  const float fr = dr * rsr, ur = fr * fr;
  const float fb = db * rsb, ub = fb * fb;
  float rho_log, lnr_jump, iblog, lnb_jump;
  if (Mth::small(ur)) {
    rho_log = half * sr * Mth::Q(ur);
    lnr_jump = 2.0f * fr * Mth::A(ur);
  } else {
    lnr_jump = Mth::ljump(Pp.rho, M.rho, dr);
    rho_log = dr / lnr_jump;
  }
  if (Mth::small(ub)) {
    const float Ab = Mth::A(ub);
    iblog = 2.0f * rsb * Ab;
    lnb_jump = 2.0f * fb * Ab;
  } else {
    lnb_jump = Mth::ljump(Pp.b, M.b, db);
    iblog = lnb_jump / db;
  }
  const float u0 = half * (M.u0 + Pp.u0), u1 = half * (M.u1 + Pp.u1), u2 = half * (M.u2 + Pp.u2);
  const float un = u0 * n0 + u1 * n1 + u2 * n2;
  const float pt = sr * rsb * half;
  const float ptp = J.ptp;
  const float uu = M.u0 * Pp.u0 + M.u1 * Pp.u1 + M.u2 * Pp.u2;
  const float Fr = rho_log * un;
  F[0] = Fr;
  F[1] = Fr * u0 + ptp * n0;
  F[2] = Fr * u1 + ptp * n1;
  F[3] = Fr * u2 + ptp * n2;
  F[4] = Fr * (iblog * half * igm1 + half * uu + phi) + pt * un;
  if (!dissipation) return;
  dissipate_bg(phi, n0, n1, n2, gamma, igm1, igamma, J, Mth::small(ur), rsr, ur, lnr_jump,
               lnb_jump, rho_log, pt, u0, u1, u2, un, F);
}

// A moving background (a flow carried by the background, continuous across
// faces and tangential at walls): the face flux's background part is the
// Euler flux f(q_bg).n, so the kernel stores F* - f(q_bg).n.  With primes for
// state minus background, {{.}} the two-side average and un = {{u}}.n:
//   F^rho - f^rho_bg = (<rho>_log - rho_bg) un + rho_bg {{u'}}.n,
//     <rho>_log - rho_bg = {{rho'}} Q(u) + rho_bg (Q(u) - 1)   (series branch),
//   F^m - f^m_bg     = (F^rho - f^rho_bg) {{u}} + f^rho_bg {{u'}} + (p* - p_bg) n,
//   F^E - f^E_bg     = (F^rho - f^rho_bg) W + f^rho_bg W' + (p* - p_bg) un + p_bg {{u'}}.n,
// W = 1/(2 (gamma-1) <b>_log) + u-.u+/2 + phi, W' = (1/<b>_log - 1/b_bg)/(2 (gamma-1))
// + (u-'.u+ + u_bg.u+')/2 and 1/<b>_log - 1/b_bg = ((A(u) - 1) - {{b'}}/b_bg)/{{b}}
// (series branch).  The dissipation is that of face_flux_bg (jumps only).
struct BgMove {
  float rb, ibb, pb;                   // background rho, 1/b, p at the node
  float ub0, ub1, ub2;                 // background velocity
  float vm0, vm1, vm2, vp0, vp1, vp2;  // u' = u - u_bg on the two sides
  float rpbar, bpbar;                  // {{rho'}}, {{b'}}
};

__device__ __forceinline__ void face_flux_bgm(const Side<float>& M, const Side<float>& Pp,
                                              float phi, float n0, float n1, float n2, float gamma,
                                              float igm1, float igamma, int dissipation,
                                              const BgFace& J, const BgMove& G, float* F) {
  using Mth = FaceMath<float>;
  const float half = 0.5f;
  const float sr = Pp.rho + M.rho, dr = J.dr;
  const float sb = Pp.b + M.b, db = J.db;
  const float rsr = Mth::rcp(sr), rsb = Mth::rcp(sb);
  const float fr = dr * rsr, ur = fr * fr;
  const float fb = db * rsb, ub = fb * fb;
  float rho_log, lnr_jump, iblog, lnb_jump, rlp, ibp;
  if (Mth::small(ur)) {
    const float Qr = Mth::Q(ur);
    rho_log = half * sr * Qr;
    lnr_jump = 2.0f * fr * Mth::A(ur);
    // Q(u) - 1 = u (-1/3 - 4u/45 - 44u^2/945)
    const float qm1 = ur * fmaf(ur, fmaf(ur, -44.0f / 945.0f, -4.0f / 45.0f), -1.0f / 3.0f);
    rlp = fmaf(G.rpbar, Qr, G.rb * qm1);
  } else {
    lnr_jump = Mth::ljump(Pp.rho, M.rho, dr);
    rho_log = dr / lnr_jump;
    rlp = rho_log - G.rb;
  }
  if (Mth::small(ub)) {
    const float Ab = Mth::A(ub);
    iblog = 2.0f * rsb * Ab;
    lnb_jump = 2.0f * fb * Ab;
    // A(u) - 1 = u (1/3 + u/5 + u^2/7)
    const float am1 = ub * fmaf(ub, fmaf(ub, 1.0f / 7.0f, 0.2f), 1.0f / 3.0f);
    ibp = 2.0f * rsb * fmaf(-G.bpbar, G.ibb, am1);
  } else {
    lnb_jump = Mth::ljump(Pp.b, M.b, db);
    iblog = lnb_jump / db;
    ibp = iblog - G.ibb;
  }
  const float u0 = half * (M.u0 + Pp.u0), u1 = half * (M.u1 + Pp.u1), u2 = half * (M.u2 + Pp.u2);
  const float v0 = half * (G.vm0 + G.vp0), v1 = half * (G.vm1 + G.vp1), v2 = half * (G.vm2 + G.vp2);
  const float un = u0 * n0 + u1 * n1 + u2 * n2;
  const float unp = v0 * n0 + v1 * n1 + v2 * n2;
  const float unb = G.ub0 * n0 + G.ub1 * n1 + G.ub2 * n2;
  const float pt = sr * rsb * half;
  const float ptp = J.ptp;
  const float uu = M.u0 * Pp.u0 + M.u1 * Pp.u1 + M.u2 * Pp.u2;
  const float uup = G.vm0 * Pp.u0 + G.vm1 * Pp.u1 + G.vm2 * Pp.u2 +
                    (G.ub0 * G.vp0 + G.ub1 * G.vp1 + G.ub2 * G.vp2);
  const float Frp = rlp * un + G.rb * unp;
  const float Frb = G.rb * unb;
  F[0] = Frp;
  F[1] = Frp * u0 + Frb * v0 + ptp * n0;
  F[2] = Frp * u1 + Frb * v1 + ptp * n1;
  F[3] = Frp * u2 + Frb * v2 + ptp * n2;
  F[4] = Frp * (iblog * half * igm1 + half * uu + phi) + Frb * (ibp * half * igm1 + half * uup) +
         ptp * un + G.pb * unp;
  if (!dissipation) return;
  dissipate_bg(phi, n0, n1, n2, gamma, igm1, igamma, J, Mth::small(ur), rsr, ur, lnr_jump,
               lnb_jump, rho_log, pt, u0, u1, u2, un, F);
}

// One face node (global face-node index tid) of one mesh.  BG: 0 none, 1 a
// background at rest (bg), 2 a moving background (bg and its state bgq).
template <typename R, int N, int BG>
__device__ __forceinline__ void face_node(const EsdgGrid& g, const EsdgPhys& P,
                                          const double* __restrict__ q,
                                          const double* __restrict__ fgeo, R* __restrict__ fflux,
                                          const double* __restrict__ bg,
                                          const double* __restrict__ bgq, const double* tr_lo,
                                          const double* tr_hi, int tr_nv, int tr_bg,
                                          long long tid) {
  constexpr int Nq = N + 1, NF2 = Nq * Nq, NP = Nq * Nq * Nq;
  if (tid >= g.nfaces * NF2) return;
  const long long f = tid / NF2;
  const int fn = (int)(tid - f * NF2);
  int d = 0;
  while (d < 2 && f >= g.face_off[d + 1]) d++;
  // direction d and the two others o1 < o2 (esdg_others) as strides: elements
  // x 1, y K0, z K0 K1; nodes x 1, y Nq, z Nq^2
  const int K0 = g.K[0], K1 = g.K[1], K2 = g.K[2];
  const int Ko1 = (d == 0) ? K1 : K0, Ko2 = (d == 2) ? K1 : K2;
  const int Kd = (d == 0) ? K0 : ((d == 1) ? K1 : K2);
  const int per = (d == 0) ? g.periodic[0] : ((d == 1) ? g.periodic[1] : g.periodic[2]);
  const int sd = (d == 0) ? 1 : ((d == 1) ? K0 : K0 * K1);
  const int so1 = (d == 0) ? K0 : 1, so2 = (d == 2) ? K0 : K0 * K1;
  const int nd = (d == 0) ? 1 : ((d == 1) ? Nq : NF2);
  const int no1 = (d == 0) ? Nq : 1, no2 = (d == 2) ? Nq : NF2;
  // the face within its direction as (a, b, plane); 32-bit unsigned divisions
  // (fewer than 2^32 faces)
  const unsigned r = (unsigned)(f - g.face_off[d]);
  const unsigned r1 = r / (unsigned)Ko1;
  const int a = (int)(r - r1 * (unsigned)Ko1);
  const unsigned r2 = r1 / (unsigned)Ko2;
  const int b = (int)(r1 - r2 * (unsigned)Ko2);
  const int Pl = (int)r2;
  // elements below and above the plane (-1 at a wall or a partition's cut)
  const int et = a * so1 + b * so2;
  const int em = (Pl > 0 || per) ? et + (Pl > 0 ? Pl - 1 : Kd - 1) * sd : -1;
  const int ep = (Pl < Kd) ? et + Pl * sd : -1;
  const int nt = (fn % Nq) * no1 + (fn / Nq) * no2;
  const int nm = nt + N * nd, npn = nt;
  const double* G = fgeo + (size_t)f * 5 * NF2;
  const double n0 = G[0 * NF2 + fn], n1 = G[1 * NF2 + fn], n2 = G[2 * NF2 + fn];
  const double scale = G[3 * NF2 + fn], phi = G[4 * NF2 + fn];
  double qm[5], qp[5];
  if (em >= 0)
    for (int v = 0; v < 5; v++) qm[v] = q[((size_t)em * 5 + v) * NP + nm];
  if (ep >= 0)
    for (int v = 0; v < 5; v++) qp[v] = q[((size_t)ep * 5 + v) * NP + npn];
  // a partition's cut x plane: the outside state is the neighbour's trace
  const bool cut = d == 0 && ((em < 0 && g.remote[0]) || (ep < 0 && g.remote[1]));
  // mixed path: the background pressure of the element below the face (at a
  // partition's low cut the neighbour's, carried in its trace)
  double pbg = 0.0;
  const size_t toff = ((size_t)b * K1 + a) * tr_nv * NF2 + fn;  // d = 0: a along y, b along z
  if constexpr (BG) {
    if (cut && em < 0 && tr_lo && tr_nv == 7) pbg = tr_lo[toff + 6 * (size_t)NF2];
    else pbg = (em >= 0) ? bg[((size_t)em * 3 + 2) * NP + nm] : bg[((size_t)ep * 3 + 2) * NP + npn];
  }
  if (cut) {
    const double* t = (em < 0) ? tr_lo : tr_hi;
    double o[5];
    if (!t) {  // no trace given: the inside state
#pragma unroll
      for (int v = 0; v < 5; v++) o[v] = (em < 0) ? qp[v] : qm[v];
    } else if (tr_bg) {  // the neighbour's background at rest (as esdg_launch_background)
      const double rb = t[toff + 5 * (size_t)NF2], pb = t[toff + 6 * (size_t)NF2];
      o[0] = rb;
      o[1] = o[2] = o[3] = 0.0;
      o[4] = fma(rb, phi, pb / (P.gamma - 1.0));
    } else {
#pragma unroll
      for (int v = 0; v < 5; v++) o[v] = t[toff + (size_t)v * NF2];
    }
    if (em < 0) {
#pragma unroll
      for (int v = 0; v < 5; v++) qm[v] = o[v];
    } else {
#pragma unroll
      for (int v = 0; v < 5; v++) qp[v] = o[v];
    }
  } else if (em < 0 || ep < 0) {  // reflecting wall: mirror the existing side
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
  R F[5];
  if constexpr (BG == 2) {
    // FP64 only where the state cancels: per side rho' = rho - rho_bg,
    // m' = m - m_bg, e' = E - E_bg - phi rho' against the background at this
    // node (one element's value: the background is a function of position),
    // and the jumps of rho and rho u.  Then in FP32 per side (as prims32bgm)
    //   u' = (m' - rho' u_bg)/rho, u = u_bg + u', p' = (gamma-1)(e' - (m'.u + rho_bg u_bg.u')/2),
    //   b' = (rho' p_bg - rho_bg p')/(2 p p_bg),
    // and the jumps and pressure mean by the identities of the branch below,
    // [[p]] = [[p']] and {{p}} - p_bg = {{p'}}.
    const int eb = em >= 0 ? em : ep, nb = em >= 0 ? nm : npn;
    const double* Qb = bgq + (size_t)eb * 5 * NP + nb;
    const double rbd = Qb[0], ebd = Qb[4 * NP];
    const double mbd[3] = {Qb[NP], Qb[2 * NP], Qb[3 * NP]};
    const float rbf = esdg_d2f(rbd), pbf = esdg_d2f(pbg);
    const float ibbf = esdg_rcpf(esdg_d2f(bg[((size_t)eb * 3 + 1) * NP + nb]));
    const float irb = esdg_rcpf(rbf);
    const float ubv[3] = {esdg_d2f(mbd[0]) * irb, esdg_d2f(mbd[1]) * irb, esdg_d2f(mbd[2]) * irb};
    const float gm1f = esdg_d2f(gm1);
    float rho[2], ir[2], v[2][3], u[2][3], pp[2], pf[2], rpf[2];
#pragma unroll
    for (int sd2 = 0; sd2 < 2; sd2++) {
      const double* qs = sd2 ? qp : qm;
      const double rp = qs[0] - rbd;
      const double ep = fma(-phi, rp, qs[4] - ebd);
      rpf[sd2] = esdg_d2f(rp);
      const float epf = esdg_d2f(ep);
      rho[sd2] = esdg_d2f(qs[0]);
      ir[sd2] = esdg_rcpf(rho[sd2]);
      float mf[3];
#pragma unroll
      for (int c = 0; c < 3; c++) {
        mf[c] = esdg_d2f(qs[1 + c] - mbd[c]);
        v[sd2][c] = fmaf(-rpf[sd2], ubv[c], mf[c]) * ir[sd2];
        u[sd2][c] = ubv[c] + v[sd2][c];
      }
      const float kb = rbf * fmaf(ubv[2], v[sd2][2], fmaf(ubv[1], v[sd2][1], ubv[0] * v[sd2][0]));
      const float kep = 0.5f * fmaf(mf[2], u[sd2][2], fmaf(mf[1], u[sd2][1], fmaf(mf[0], u[sd2][0], kb)));
      pp[sd2] = gm1f * (epf - kep);
      pf[sd2] = pbf + pp[sd2];
    }
    const Side<float> M{rho[0], u[0][0], u[0][1], u[0][2], 0.5f * rho[0] * esdg_rcpf(pf[0])};
    const Side<float> Pp{rho[1], u[1][0], u[1][1], u[1][2], 0.5f * rho[1] * esdg_rcpf(pf[1])};
    const float dr = esdg_d2f(qp[0] - qm[0]);
    const float dm0 = esdg_d2f(qp[1] - qm[1]), dm1 = esdg_d2f(qp[2] - qm[2]),
                dm2 = esdg_d2f(qp[3] - qm[3]);
    const float dp = pp[1] - pp[0];
    const float rbar = 0.5f * (Pp.rho + M.rho), pbar = 0.5f * (pf[1] + pf[0]);
    const float X = fmaf(dr, pbar, -rbar * dp);  // rho+ p- - rho- p+
    BgFace J;
    J.dr = dr;
    J.db = X * esdg_rcpf(2.0f * pf[1] * pf[0]);
    const float irbar = 0.5f * (ir[1] + ir[0]), dirr = dr * ir[1] * ir[0];
    const float du0 = fmaf(dm0, irbar, -0.5f * (Pp.rho * Pp.u0 + M.rho * M.u0) * dirr);
    const float du1 = fmaf(dm1, irbar, -0.5f * (Pp.rho * Pp.u1 + M.rho * M.u1) * dirr);
    const float du2 = fmaf(dm2, irbar, -0.5f * (Pp.rho * Pp.u2 + M.rho * M.u2) * dirr);
    const float ub0 = 0.5f * (Pp.u0 + M.u0), ub1 = 0.5f * (Pp.u1 + M.u1), ub2 = 0.5f * (Pp.u2 + M.u2);
    const float bbar = 0.5f * (Pp.b + M.b);
    J.dbu0 = fmaf(J.db, ub0, bbar * du0);
    J.dbu1 = fmaf(J.db, ub1, bbar * du1);
    J.dbu2 = fmaf(J.db, ub2, bbar * du2);
    const float bu0 = 0.5f * (Pp.b * Pp.u0 + M.b * M.u0), bu1 = 0.5f * (Pp.b * Pp.u1 + M.b * M.u1),
                bu2 = 0.5f * (Pp.b * Pp.u2 + M.b * M.u2);
    J.dbuu = fmaf(J.dbu0, ub0, fmaf(J.dbu1, ub1, fmaf(J.dbu2, ub2,
                  fmaf(bu0, du0, fmaf(bu1, du1, bu2 * du2)))));
    const float D = fmaf(2.0f * rbar, pbar, -0.5f * dr * dp);
    J.ptp = fmaf(dp * X, esdg_rcpf(2.0f * D), 0.5f * (pp[1] + pp[0]));
    BgMove Gm;
    Gm.rb = rbf;
    Gm.ibb = ibbf;
    Gm.pb = pbf;
    Gm.ub0 = ubv[0];
    Gm.ub1 = ubv[1];
    Gm.ub2 = ubv[2];
    Gm.vm0 = v[0][0];
    Gm.vm1 = v[0][1];
    Gm.vm2 = v[0][2];
    Gm.vp0 = v[1][0];
    Gm.vp1 = v[1][1];
    Gm.vp2 = v[1][2];
    Gm.rpbar = 0.5f * (rpf[0] + rpf[1]);
    const float bpm = fmaf(rpf[0], pbf, -rbf * pp[0]) * esdg_rcpf(2.0f * pf[0] * pbf);
    const float bpp = fmaf(rpf[1], pbf, -rbf * pp[1]) * esdg_rcpf(2.0f * pf[1] * pbf);
    Gm.bpbar = 0.5f * (bpm + bpp);
    face_flux_bgm(M, Pp, esdg_d2f(phi), esdg_d2f(n0), esdg_d2f(n1), esdg_d2f(n2),
                  esdg_d2f(P.gamma), esdg_d2f(P.igm1), esdg_d2f(P.igamma), P.dissipation, J, Gm, F);
  } else if constexpr (BG) {
    // FP64 only where the state cancels (13 instructions): each side's pressure
    // E - rho phi - KE (KE in FP32), and the jumps of rho, rho u and p.  The
    // jumps of b, b u, b |u|^2 and the pressure mean follow from them by exact
    // identities evaluated in FP32, with ({{.}} the two-side average):
    //   [[b]] = (rho+ p- - rho- p+)/(2 p+ p-),  rho+ p- - rho- p+ = [[rho]] {{p}} - {{rho}} [[p]],
    //   [[u]] = [[rho u]] {{1/rho}} - {{rho u}} [[rho]]/(rho+ rho-),
    //   [[x y]] = [[x]] {{y}} + {{x}} [[y]]  (for b u and (b u) . u),
    //   p* - p_bg = {{p}} - p_bg + [[p]] (rho+ p- - rho- p+)/(2 D),
    //   D = rho+ p- + rho- p+ = 2 {{rho}} {{p}} - [[rho]] [[p]]/2.
    float mf[5], pf5[5];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      mf[v] = esdg_d2f(qm[v]);
      pf5[v] = esdg_d2f(qp[v]);
    }
    const float irm = esdg_rcpf(mf[0]), irp = esdg_rcpf(pf5[0]);
    const Side<float> M{mf[0], mf[1] * irm, mf[2] * irm, mf[3] * irm, 0.0f};
    Side<float> Pp{pf5[0], pf5[1] * irp, pf5[2] * irp, pf5[3] * irp, 0.0f};
    const float kem = 0.5f * fmaf(mf[3], M.u2, fmaf(mf[2], M.u1, mf[1] * M.u0));
    const float kep = 0.5f * fmaf(pf5[3], Pp.u2, fmaf(pf5[2], Pp.u1, pf5[1] * Pp.u0));
    const double prm = gm1 * (fma(-qm[0], phi, qm[4]) - esdg_f2d(kem));
    const double prp = gm1 * (fma(-qp[0], phi, qp[4]) - esdg_f2d(kep));
    const float pmf = esdg_d2f(prm), ppf = esdg_d2f(prp);
    Side<float> Mb = M;
    Mb.b = 0.5f * M.rho * esdg_rcpf(pmf);
    Pp.b = 0.5f * Pp.rho * esdg_rcpf(ppf);
    const float dr = esdg_d2f(qp[0] - qm[0]);
    const float dm0 = esdg_d2f(qp[1] - qm[1]), dm1 = esdg_d2f(qp[2] - qm[2]),
                dm2 = esdg_d2f(qp[3] - qm[3]);
    const float dp = esdg_d2f(prp - prm);
    const float pbar_p = esdg_d2f(esdg_ldexp(prp + prm, -1) - pbg);  // {{p}} - p_bg
    const float rbar = 0.5f * (Pp.rho + Mb.rho), pbar = 0.5f * (ppf + pmf);
    const float X = fmaf(dr, pbar, -rbar * dp);  // rho+ p- - rho- p+
    BgFace J;
    J.dr = dr;
    J.db = X * esdg_rcpf(2.0f * ppf * pmf);
    const float irbar = 0.5f * (irp + irm), dirr = dr * irp * irm;
    const float du0 = fmaf(dm0, irbar, -0.5f * (pf5[1] + mf[1]) * dirr);
    const float du1 = fmaf(dm1, irbar, -0.5f * (pf5[2] + mf[2]) * dirr);
    const float du2 = fmaf(dm2, irbar, -0.5f * (pf5[3] + mf[3]) * dirr);
    const float ub0 = 0.5f * (Pp.u0 + Mb.u0), ub1 = 0.5f * (Pp.u1 + Mb.u1), ub2 = 0.5f * (Pp.u2 + Mb.u2);
    const float bbar = 0.5f * (Pp.b + Mb.b);
    J.dbu0 = fmaf(J.db, ub0, bbar * du0);
    J.dbu1 = fmaf(J.db, ub1, bbar * du1);
    J.dbu2 = fmaf(J.db, ub2, bbar * du2);
    const float bu0 = 0.5f * (Pp.b * Pp.u0 + Mb.b * Mb.u0), bu1 = 0.5f * (Pp.b * Pp.u1 + Mb.b * Mb.u1),
                bu2 = 0.5f * (Pp.b * Pp.u2 + Mb.b * Mb.u2);
    J.dbuu = fmaf(J.dbu0, ub0, fmaf(J.dbu1, ub1, fmaf(J.dbu2, ub2,
                  fmaf(bu0, du0, fmaf(bu1, du1, bu2 * du2)))));
    const float D = fmaf(2.0f * rbar, pbar, -0.5f * dr * dp);
    J.ptp = fmaf(dp * X, esdg_rcpf(2.0f * D), pbar_p);
    face_flux_bg(Mb, Pp, esdg_d2f(phi), esdg_d2f(n0), esdg_d2f(n1), esdg_d2f(n2), esdg_d2f(P.gamma),
                 esdg_d2f(P.igm1), esdg_d2f(P.igamma), P.dissipation, J, F);
  } else {
    const Side<R> M = side_from<R>(qm, phi, gm1), Pp = side_from<R>(qp, phi, gm1);
    face_flux<R>(M, Pp, to_r<R>(phi), to_r<R>(n0), to_r<R>(n1), to_r<R>(n2), to_r<R>(P.gamma),
                 to_r<R>(P.igm1), to_r<R>(P.igamma), P.dissipation, F);
  }
  R* out = fflux + (size_t)f * 5 * NF2;
  const R sc = to_r<R>(scale);
#pragma unroll
  for (int v = 0; v < 5; v++) out[v * NF2 + fn] = sc * F[v];
}

// Face of work item w when a launch covers every face: layer by layer in z
// (element layer k: its x faces, its y faces, then the z plane below it; the
// z planes past the last layer at the end), so that the few megabytes of
// state a layer's faces read stay in L2 for all three directions instead of
// streaming the whole state through L2 once per direction (the face ids,
// and with them the flux layout, are unchanged).
// Face indices fit in 32 bits (es_dg_create admits at most 2^30 elements, so
// fewer than 2^32 faces): the divisions by runtime extents are 32-bit unsigned
// ones, several times cheaper than 64-bit divisions on an issue-bound kernel.
__device__ __forceinline__ long long face_layered(const EsdgGrid& g, long long w64) {
  const unsigned w = (unsigned)w64;
  const unsigned K0 = g.K[0], K1 = g.K[1], K2 = g.K[2];
  const unsigned nx = (unsigned)g.nplanes[0] * K1, ny = (unsigned)g.nplanes[1] * K0;
  const unsigned L = nx + ny + K0 * K1;
  if (w >= K2 * L) return g.face_off[2] + (long long)K2 * K1 * K0 + (w - K2 * L);
  const unsigned k = w / L;
  unsigned r = w - k * L;
  if (r < nx) {
    const unsigned P = r / K1;
    return g.face_off[0] + ((long long)P * K2 + k) * K1 + (r - P * K1);
  }
  r -= nx;
  if (r < ny) {
    const unsigned P = r / K0;
    return g.face_off[1] + ((long long)P * K2 + k) * K0 + (r - P * K0);
  }
  r -= ny;
  const unsigned b = r / K0;
  return g.face_off[2] + ((long long)k * K1 + b) * K0 + (r - b * K0);
}

// mixed: at most 64 registers, four 256-thread CTAs per SM
template <typename R, int N, int BG>
__global__ void __launch_bounds__(256, sizeof(R) == sizeof(float) ? 4 : 1)
    k_face(EsdgGrid g, EsdgPhys P, const double* __restrict__ q,
                                              const double* __restrict__ fgeo,
                                              R* __restrict__ fflux,
                                              const double* __restrict__ bg, EsdgTraces tr,
                                              const double* __restrict__ bgq, long long t0,
                                              long long t1) {
  // face nodes t0 .. t1 - 1 (global face-node indices); a launch over every
  // face takes them in the layered order
  constexpr long long NF2 = (N + 1) * (N + 1);
  long long tid = t0 + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= t1) return;
  if (t0 == 0 && t1 == g.nfaces * NF2) {
    const long long w = tid / NF2;
    tid = face_layered(g, w) * NF2 + (tid - w * NF2);
  }
  face_node<R, N, BG>(g, P, q, fgeo, fflux, bg, bgq, tr.lo, tr.hi, tr.nv, tr.bgmode, tid);
}

// A partition's traces: one thread per (side, face of the plane, face node);
// with a background (nv = 7) also its rho_bg and p_bg.
__global__ void k_trace_pack(EsdgGrid g, const double* __restrict__ q,
                             const double* __restrict__ bg, int nv, double* __restrict__ lo,
                             double* __restrict__ hi) {
  const int Nq = g.Nq, NF2 = Nq * Nq, np = g.np;
  const long long per_side = (long long)g.K[1] * g.K[2] * NF2;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= 2 * per_side) return;
  const int side = (int)(tid / per_side);
  const long long r = tid - side * per_side;
  double* out = side ? hi : lo;
  if (!out) return;
  const long long j = r / NF2;  // face of the plane: a + K[1] b
  const int fn = (int)(r - j * NF2);
  const int a = (int)(j % g.K[1]), b = (int)(j / g.K[1]);
  const int ex = side ? g.K[0] - 1 : 0;
  const long long e = ex + (long long)g.K[0] * (a + (long long)g.K[1] * b);
  const int n = esdg_node(Nq, side ? g.N : 0, fn % Nq, fn / Nq);
  for (int v = 0; v < 5; v++)
    out[(j * nv + v) * NF2 + fn] = q[((size_t)e * 5 + v) * np + n];
  if (bg && nv == 7) {
    out[(j * nv + 5) * NF2 + fn] = bg[((size_t)e * 3 + 0) * np + n];
    out[(j * nv + 6) * NF2 + fn] = bg[((size_t)e * 3 + 2) * np + n];
  }
}

// Persistent batched face kernel: CTAs of 256 threads stride over a work table
// of (member, first face node) tiles of meshes with the same N and precision.
template <typename R, int N, bool BG>
__global__ void __launch_bounds__(256) k_face_batch(const EsdgMember* __restrict__ members,
                                                    const int2* __restrict__ tiles,
                                                    const int* __restrict__ ntiles) {
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
    // the member's faces in the layered order (a table covers all of them)
    constexpr long long NF2 = (N + 1) * (N + 1);
    long long tid = (long long)tile.y + threadIdx.x;
    if (tid < mb.g.nfaces * NF2) {
      const long long w = tid / NF2;
      tid = face_layered(mb.g, w) * NF2 + (tid - w * NF2);
    }
    face_node<R, N, BG>(mb.g, mb.P, mb.a.q_in, mb.fgeo, (R*)mb.a.fflux, mb.bg, nullptr,
                        nullptr, nullptr, 5, 0, tid);
    __syncthreads();
  }
}

template <typename R, int BG>
cudaError_t launch_face_t(const EsdgGrid& g, const EsdgPhys& P, const double* q, const double* fgeo,
                          R* fflux, const double* bg, EsdgTraces tr, cudaStream_t s,
                          const double* bgq, long long f0, long long f1) {
  const long long nf2 = (long long)g.Nq * g.Nq;
  if (f1 < 0 || f1 > g.nfaces) f1 = g.nfaces;
  if (f0 < 0) f0 = 0;
  if (f1 <= f0) return cudaSuccess;
  const long long t0 = f0 * nf2, t1 = f1 * nf2;
  const unsigned blocks = (unsigned)((t1 - t0 + 255) / 256);
  switch (g.N) {
    case 1: k_face<R, 1, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 2: k_face<R, 2, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 3: k_face<R, 3, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 4: k_face<R, 4, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 5: k_face<R, 5, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 6: k_face<R, 6, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    case 7: k_face<R, 7, BG><<<blocks, 256, 0, s>>>(g, P, q, fgeo, fflux, bg, tr, bgq, t0, t1); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t esdg_launch_face_batch(int N, int mixed, int bg, const EsdgMember* members,
                                   const int2* tiles, const int* ntiles, int grid, cudaStream_t s) {
#define ESDG_FB(NN)                                                                        \
  case NN:                                                                                 \
    if (mixed && bg) k_face_batch<float, NN, true><<<grid, 256, 0, s>>>(members, tiles, ntiles);  \
    else if (mixed) k_face_batch<float, NN, false><<<grid, 256, 0, s>>>(members, tiles, ntiles);  \
    else k_face_batch<double, NN, false><<<grid, 256, 0, s>>>(members, tiles, ntiles);      \
    break;
  switch (N) {
    ESDG_FB(1) ESDG_FB(2) ESDG_FB(3) ESDG_FB(4) ESDG_FB(5) ESDG_FB(6) ESDG_FB(7)
    default: return cudaErrorInvalidValue;
  }
#undef ESDG_FB
  return cudaGetLastError();
}

cudaError_t esdg_launch_face(const EsdgGrid& g, const EsdgPhys& P, int mixed, const double* q,
                             const double* fgeo, void* fflux, cudaStream_t s, const double* bg,
                             EsdgTraces tr, const double* bgq, long long f0, long long f1) {
  if (mixed && bg && bgq)
    return launch_face_t<float, 2>(g, P, q, fgeo, (float*)fflux, bg, tr, s, bgq, f0, f1);
  if (mixed && bg)
    return launch_face_t<float, 1>(g, P, q, fgeo, (float*)fflux, bg, tr, s, nullptr, f0, f1);
  if (mixed)
    return launch_face_t<float, 0>(g, P, q, fgeo, (float*)fflux, nullptr, tr, s, nullptr, f0, f1);
  return launch_face_t<double, 0>(g, P, q, fgeo, (double*)fflux, nullptr, tr, s, nullptr, f0, f1);
}

cudaError_t esdg_launch_trace_pack(const EsdgGrid& g, const double* q, const double* bg, int nv,
                                   double* send_lo, double* send_hi, cudaStream_t s) {
  const long long nt = 2LL * g.K[1] * g.K[2] * g.Nq * g.Nq;
  if ((!send_lo && !send_hi) || nt == 0) return cudaSuccess;
  if (nv != 5 && nv != 7) return cudaErrorInvalidValue;
  k_trace_pack<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, q, bg, nv, send_lo, send_hi);
  return cudaGetLastError();
}
