// volume_impl.cuh -- flux-differencing volume kernel (Section 3, the volume term
// of Eq. (nm:semi), with the optimisations of Section 4.1).
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
#include <cstring>
#include <type_traits>

#include "esdg_internal.cuh"

namespace esdg_vol {

template <int N, bool MIXED>
struct Cfg;
// elements per CTA, chosen so that 3 Nq^2 EPB pencils fill whole warps
template <> struct Cfg<1, false> { static constexpr int EPB = 8; };
template <> struct Cfg<2, false> { static constexpr int EPB = 16; };
template <> struct Cfg<3, false> { static constexpr int EPB = 8; };
template <> struct Cfg<4, false> { static constexpr int EPB = 5; };
template <> struct Cfg<5, false> { static constexpr int EPB = 2; };
template <> struct Cfg<6, false> { static constexpr int EPB = 1; };
template <> struct Cfg<7, false> { static constexpr int EPB = 1; };
template <> struct Cfg<1, true> { static constexpr int EPB = 16; };
template <> struct Cfg<2, true> { static constexpr int EPB = 16; };
template <> struct Cfg<3, true> { static constexpr int EPB = 8; };
template <> struct Cfg<4, true> { static constexpr int EPB = 5; };
template <> struct Cfg<5, true> { static constexpr int EPB = 3; };
template <> struct Cfg<6, true> { static constexpr int EPB = 2; };
template <> struct Cfg<7, true> { static constexpr int EPB = 2; };

template <int N, bool MIXED, bool BG = false, int EPB_ = 0>
struct Shape {
  static constexpr int Nq = N + 1, NP = Nq * Nq * Nq, NPEN = Nq * Nq;
  static constexpr int EPB = EPB_ > 0 ? EPB_ : Cfg<N, MIXED>::EPB;  // elements per CTA (tile)
  static constexpr int PENCILS = 3 * NPEN * EPB;
  static constexpr int THREADS = ((PENCILS + 31) / 32) * 32;
  // node fields: rq=rho/4, bh=b/2, ib=1/b, uh=u/2 (3), ph=phi/2, [lr, lb], nh=Ja/2 (9),
  // [background: rq'=rho'/4, bh'=b'/2, rq_bg, bh_bg, 1/b_bg, p_bg, p'=p-p_bg]
  static constexpr int F_LR = 7, F_LB = 8;
  static constexpr int F_NH = MIXED ? 7 : 9;
  static constexpr int F_BG = F_NH + 9;
  static constexpr int NF = F_NH + 9 + (BG ? 7 : 0);
  using R = typename std::conditional<MIXED, float, double>::type;
  static constexpr size_t SMEM = sizeof(R) * (size_t)NF * NP * EPB;
};

template <typename R>
struct Node {
  R rq, bh, ib, u0, u1, u2, ph, n0, n1, n2, lr, lb;
  R rqp, bhp, rqb, bhb, ibb, pb, pp;  // perturbation and background (mixed mode with a background)
};

template <typename R, bool LOGS, int F_NH, int NP, bool BG = false>
__device__ __forceinline__ Node<R> load_node(const R* __restrict__ S, int n, int d) {
  Node<R> a;
  a.rq = S[0 * NP + n];
  a.bh = S[1 * NP + n];
  a.ib = S[2 * NP + n];
  a.u0 = S[3 * NP + n];
  a.u1 = S[4 * NP + n];
  a.u2 = S[5 * NP + n];
  a.ph = S[6 * NP + n];
  const R* nh = S + (F_NH + 3 * d) * NP;
  a.n0 = nh[0 * NP + n];
  a.n1 = nh[1 * NP + n];
  a.n2 = nh[2 * NP + n];
  if (LOGS && F_NH == 9) {
    a.lr = S[7 * NP + n];
    a.lb = S[8 * NP + n];
  } else {
    a.lr = a.lb = (R)0;
  }
  if (BG) {
    const R* b = S + (F_NH + 9) * NP;
    a.rqp = b[0 * NP + n];
    a.bhp = b[1 * NP + n];
    a.rqb = b[2 * NP + n];
    a.bhb = b[3 * NP + n];
    a.ibb = b[4 * NP + n];
    a.pb = b[5 * NP + n];
    a.pp = b[6 * NP + n];
  }
  return a;
}

// The artanh series of 1/<b>_log scaled by ce = 1/(2(gamma - 1)): the energy
// flux only needs ce/<b>_log, so ce goes into the coefficients (computed once
// per thread) and one FMA per pair folds the term into the energy bracket.
// Tail beyond u^1 in FP32 (see esdg_A_t).
struct CeSeries {
  double c0, c1;    // ce, ce/3
  float c2f, c3f;   // ce/5, ce/7
};
__device__ __forceinline__ CeSeries ce_series(double ce) {
  return CeSeries{ce, ce * (1.0 / 3.0), esdg_d2f(ce * 0.2), esdg_d2f(ce * (1.0 / 7.0))};
}
__device__ __forceinline__ double esdg_Ace_t(double u, const CeSeries& c) {
  const float tail = fmaf(esdg_d2f_tail(u), c.c3f, c.c2f);
  return fma(u, fma(u, esdg_f2d_pos(tail), c.c1), c.c0);
}

// One unordered pair (i = A, l = B) in FP64: 61 FP64 instructions on the
// series path.  ai += Dt_il H(i,l), al += Dt_li H(l,i).  The momentum flux is
// regrouped as Fr {{u}} + (p* + g_own) {{n}}, so the gravity coefficient of
// each side folds into its pressure term with one FMA.
template <bool LOGS>
__device__ __forceinline__ void pair64(const Node<double>& A, const Node<double>& B, double dil,
                                       double dli, const CeSeries& cs, double* ai, double* al) {
  const double sr = A.rq + B.rq;  // {{rho}}/2
  const double sb = A.bh + B.bh;  // {{b}}
  const double rsb = esdg_rcp(sb);
  const double pt = sr * rsb;     // p* = {{rho}}/(2{{b}})
  const double dr = A.rq - B.rq, db = A.bh - B.bh;
  const double fr = dr * esdg_rcp_lo(sr), ur = fr * fr;
  const double fb = db * rsb, ub = fb * fb;
  const double uu = fma(A.u2, B.u2, fma(A.u1, B.u1, A.u0 * B.u0));  // u_i . u_l / 4
  const double t = fma(2.0, uu, A.ph + B.ph);                        // u_i.u_l/2 + {{phi}}
  double rlog, bracket;  // <rho>_log and ce/<b>_log + t
  if (!LOGS) {
    rlog = sr * esdg_Q2_t(ur);
    bracket = fma(rsb, esdg_Ace_t(ub, cs), t);
  } else {
    if (esdg_lt_pos(ur, ESDG_LOG_EPS)) rlog = sr * esdg_Q2_t(ur);
    else rlog = (4.0 * dr) * esdg_rcp(A.lr - B.lr);
    if (esdg_lt_pos(ub, ESDG_LOG_EPS)) bracket = fma(rsb, esdg_Ace_t(ub, cs), t);
    else bracket = fma((A.lb - B.lb) * esdg_rcp(2.0 * db), cs.c0, t);
  }
  const double n0 = A.n0 + B.n0, n1 = A.n1 + B.n1, n2 = A.n2 + B.n2;  // {{Ja^d}}
  const double u0 = A.u0 + B.u0, u1 = A.u1 + B.u1, u2 = A.u2 + B.u2;  // {{u}}
  const double un = fma(u2, n2, fma(u1, n1, u0 * n0));
  const double Fr = rlog * un;
  const double f0 = Fr * u0, f1 = Fr * u1, f2 = Fr * u2;
  const double FE = un * fma(rlog, bracket, pt);
  // gravity: 1/2 rho_hat [[phi]] with rho_hat = {{b}} <rho>_log / b_(own node)
  const double gq = sb * rlog * (B.ph - A.ph);
  const double pi = fma(gq, A.ib, pt), pl = fma(-gq, B.ib, pt);
  ai[0] = fma(dil, Fr, ai[0]);
  ai[1] = fma(dil, fma(pi, n0, f0), ai[1]);
  ai[2] = fma(dil, fma(pi, n1, f1), ai[2]);
  ai[3] = fma(dil, fma(pi, n2, f2), ai[3]);
  ai[4] = fma(dil, FE, ai[4]);
  al[0] = fma(dli, Fr, al[0]);
  al[1] = fma(dli, fma(pl, n0, f0), al[1]);
  al[2] = fma(dli, fma(pl, n1, f1), al[2]);
  al[3] = fma(dli, fma(pl, n2, f2), al[3]);
  al[4] = fma(dli, FE, al[4]);
}

// The same pair in FP32 (mixed mode; geopotential relative to the element).
template <bool LOGS>
__device__ __forceinline__ void pair32(const Node<float>& A, const Node<float>& B, float dil,
                                       float dli, float ce, float* ai, float* al) {
  const float sr = A.rq + B.rq;
  const float sb = A.bh + B.bh;
  const float rsb = esdg_rcpf(sb);
  const float pt = sr * rsb;
  const float dr = A.rq - B.rq, db = A.bh - B.bh;
  const float fr = dr * esdg_rcpf(sr), ur = fr * fr;
  const float fb = db * rsb, ub = fb * fb;
  float rlog, iblog;
  if (!LOGS || (ur < ESDG_LOG_EPS32 && ub < ESDG_LOG_EPS32)) {
    rlog = sr * esdg_Q2f(ur);
    iblog = rsb * esdg_Af(ub);
  } else {
    rlog = (ur < ESDG_LOG_EPS32) ? sr * esdg_Q2f(ur)
                                 : (4.0f * dr) / log1pf(dr * esdg_rcpf(B.rq));
    iblog = (ub < ESDG_LOG_EPS32) ? rsb * esdg_Af(ub)
                                  : log1pf(db * esdg_rcpf(B.bh)) / (2.0f * db);
  }
  const float n0 = A.n0 + B.n0, n1 = A.n1 + B.n1, n2 = A.n2 + B.n2;
  const float u0 = A.u0 + B.u0, u1 = A.u1 + B.u1, u2 = A.u2 + B.u2;
  const float un = fmaf(u2, n2, fmaf(u1, n1, u0 * n0));
  const float Fr = rlog * un;
  const float m0 = fmaf(Fr, u0, pt * n0);
  const float m1 = fmaf(Fr, u1, pt * n1);
  const float m2 = fmaf(Fr, u2, pt * n2);
  const float uu = fmaf(A.u2, B.u2, fmaf(A.u1, B.u1, A.u0 * B.u0));
  const float t = fmaf(2.0f, uu, A.ph + B.ph);
  const float FE = fmaf(Fr, fmaf(iblog, ce, t), pt * un);
  const float gq = sb * rlog * (B.ph - A.ph);
  const float gi = gq * A.ib, gl = -gq * B.ib;
  ai[0] = fmaf(dil, Fr, ai[0]);
  ai[1] = fmaf(dil, fmaf(gi, n0, m0), ai[1]);
  ai[2] = fmaf(dil, fmaf(gi, n1, m1), ai[2]);
  ai[3] = fmaf(dil, fmaf(gi, n2, m2), ai[3]);
  ai[4] = fmaf(dil, FE, ai[4]);
  al[0] = fmaf(dli, Fr, al[0]);
  al[1] = fmaf(dli, fmaf(gl, n0, m0), al[1]);
  al[2] = fmaf(dli, fmaf(gl, n1, m1), al[2]);
  al[3] = fmaf(dli, fmaf(gl, n2, m2), al[3]);
  al[4] = fmaf(dli, FE, al[4]);
}

// The FP32 pair relative to a hydrostatic background (u_bg = 0): the
// momentum flux's pressure and gravity parts are formed as exact differences
// H - H_bg in perturbation variables rho' = rho - rho_bg, b' = b - b_bg, so
// their FP32 rounding is relative to the perturbation, not to the hydrostatic
// pressure (the background's own FP64 right-hand side is added in the
// epilogue).  The pressure mean is rewritten exactly as
//   p* = {{rho}}/(2{{b}}) = {{p}} + T,  T = (p_i - p_l)(rho_i p_l - rho_l p_i) / (2 D),
//   D = rho_i p_l + rho_l p_i,
// so p* - p*_bg = {{p'}} + T - T_bg with p' = p - p_bg exact from the FP64
// prologue and T - T_bg expanded into terms that each carry a perturbation
// factor.  With sums over the pair (sr = rq_i + rq_l etc.):
//   <rho>_log - <rho_bg>_log = sr' Q2(u) + sr_bg (u - u_bg) S2(u, u_bg),
//     u - u_bg = (f - f_bg)(f + f_bg), f - f_bg = 2 (rq'_i rq_bg,l - rq'_l rq_bg,i)/(sr sr_bg),
//     S2 the divided difference of the Q2 polynomial,
//   {{b}}/b_i - {{b_bg}}/b_bg,i = 2 (bh'_l bh_bg,i - bh_bg,l bh'_i) / (b_i b_bg,i),
// and the gravity difference follows by the product rule.  Density and energy
// fluxes carry no background part (u_bg = 0) and are unchanged.
template <bool LOGS>
__device__ __forceinline__ void pair32bg(const Node<float>& A, const Node<float>& B, float dil,
                                         float dli, float ce, float* ai, float* al) {
  const float sr = A.rq + B.rq;
  const float sb = A.bh + B.bh;
  const float rsb = esdg_rcpf(sb);
  const float pt = sr * rsb;
  const float dr = A.rq - B.rq, db = A.bh - B.bh;
  const float rsr = esdg_rcpf(sr);
  const float fr = dr * rsr, ur = fr * fr;
  const float fb = db * rsb, ub = fb * fb;
  // background sums and perturbation sums
  const float srb = A.rqb + B.rqb, sbb = A.bhb + B.bhb;
  const float srp = A.rqp + B.rqp;
  float ptp;
  {
    const float ri = 4.0f * A.rqb, rl = 4.0f * B.rqb, rpi = 4.0f * A.rqp, rpl = 4.0f * B.rqp;
    const float dpb = A.pb - B.pb, dpp = A.pp - B.pp;
    const float Cb = ri * B.pb - rl * A.pb;
    const float Db = fmaf(ri, B.pb, rl * A.pb);
    const float x1 = fmaf(ri, B.pp, fmaf(rpi, B.pb, rpi * B.pp));
    const float x2 = fmaf(rl, A.pp, fmaf(rpl, A.pb, rpl * A.pp));
    const float Cp = x1 - x2, Dp = x1 + x2;
    const float C = Cb + Cp, D = Db + Dp;
    const float num = fmaf(dpp * C, Db, dpb * fmaf(Cp, Db, -Cb * Dp));
    ptp = fmaf(0.5f, A.pp + B.pp, num * esdg_rcpf(2.0f * D * Db));
  }
  const float drb = A.rqb - B.rqb;
  const float rsrb = esdg_rcpf(srb);
  const float frb = drb * rsrb, urb = frb * frb;
  float rlog, iblog, rlogp;
  if (!LOGS || (ur < ESDG_LOG_EPS32 && ub < ESDG_LOG_EPS32 && urb < ESDG_LOG_EPS32)) {
    const float q2 = esdg_Q2f(ur);
    rlog = sr * q2;
    iblog = rsb * esdg_Af(ub);
    const float fdiff = 2.0f * (A.rqp * B.rqb - B.rqp * A.rqb) * rsr * rsrb;
    const float udiff = fdiff * (fr + frb);
    // divided difference of Q2(u) = 2 - 2u/3 - 8u^2/45 - 88u^3/945
    const float s2 = fmaf(-88.0f / 945.0f, fmaf(ur, ur, fmaf(ur, urb, urb * urb)),
                          fmaf(-8.0f / 45.0f, ur + urb, -2.0f / 3.0f));
    rlogp = fmaf(srp, q2, srb * udiff * s2);
  } else {
    rlog = (ur < ESDG_LOG_EPS32) ? sr * esdg_Q2f(ur)
                                 : (4.0f * dr) / log1pf(dr * esdg_rcpf(B.rq));
    iblog = (ub < ESDG_LOG_EPS32) ? rsb * esdg_Af(ub)
                                  : log1pf(db * esdg_rcpf(B.bh)) / (2.0f * db);
    const float rlogb = (urb < ESDG_LOG_EPS32) ? srb * esdg_Q2f(urb)
                                               : (4.0f * drb) / log1pf(drb * esdg_rcpf(B.rqb));
    rlogp = rlog - rlogb;
  }
  const float n0 = A.n0 + B.n0, n1 = A.n1 + B.n1, n2 = A.n2 + B.n2;
  const float u0 = A.u0 + B.u0, u1 = A.u1 + B.u1, u2 = A.u2 + B.u2;
  const float un = fmaf(u2, n2, fmaf(u1, n1, u0 * n0));
  const float Fr = rlog * un;
  const float m0 = fmaf(Fr, u0, ptp * n0);
  const float m1 = fmaf(Fr, u1, ptp * n1);
  const float m2 = fmaf(Fr, u2, ptp * n2);
  const float uu = fmaf(A.u2, B.u2, fmaf(A.u1, B.u1, A.u0 * B.u0));
  const float t = fmaf(2.0f, uu, A.ph + B.ph);
  const float FE = fmaf(Fr, fmaf(iblog, ce, t), pt * un);
  // gravity perturbation
  const float dph = B.ph - A.ph;
  const float dYi = 2.0f * (B.bhp * A.bhb - B.bhb * A.bhp) * A.ib * A.ibb;
  const float dYl = 2.0f * (A.bhp * B.bhb - A.bhb * B.bhp) * B.ib * B.ibb;
  const float gi = dph * fmaf(dYi, rlog, sbb * A.ibb * rlogp);
  const float gl = -dph * fmaf(dYl, rlog, sbb * B.ibb * rlogp);
  ai[0] = fmaf(dil, Fr, ai[0]);
  ai[1] = fmaf(dil, fmaf(gi, n0, m0), ai[1]);
  ai[2] = fmaf(dil, fmaf(gi, n1, m1), ai[2]);
  ai[3] = fmaf(dil, fmaf(gi, n2, m2), ai[3]);
  ai[4] = fmaf(dil, FE, ai[4]);
  al[0] = fmaf(dli, Fr, al[0]);
  al[1] = fmaf(dli, fmaf(gl, n0, m0), al[1]);
  al[2] = fmaf(dli, fmaf(gl, n1, m1), al[2]);
  al[3] = fmaf(dli, fmaf(gl, n2, m2), al[3]);
  al[4] = fmaf(dli, FE, al[4]);
}

// ce: 1/(2(gamma - 1)) as float (mixed) or as the scaled series (FP64)
template <int N, bool MIXED, bool LOGS, bool BG, typename CE>
__device__ __forceinline__ void pencil_pass(const typename Shape<N, MIXED, BG>::R* __restrict__ S,
                                            int d, int base, int stride, const EsdgLGL& L,
                                            const CE& ce,
                                            typename Shape<N, MIXED, BG>::R (&acc)[N + 1][5]) {
  using SH = Shape<N, MIXED, BG>;
  using R = typename SH::R;
  constexpr int Nq = N + 1;
#pragma unroll
  for (int i = 0; i < Nq; i++) {
    const Node<R> A = load_node<R, LOGS, SH::F_NH, SH::NP, BG>(S, base + i * stride, d);
#pragma unroll
    for (int l = i + 1; l < Nq; l++) {
      const Node<R> B = load_node<R, LOGS, SH::F_NH, SH::NP, BG>(S, base + l * stride, d);
      if constexpr (MIXED && BG)
        pair32bg<LOGS>(A, B, L.Dtf[i][l], L.Dtf[l][i], ce, acc[i], acc[l]);
      else if constexpr (MIXED)
        pair32<LOGS>(A, B, L.Dtf[i][l], L.Dtf[l][i], ce, acc[i], acc[l]);
      else
        pair64<LOGS>(A, B, L.Dt[i][l], L.Dt[l][i], ce, acc[i], acc[l]);
    }
  }
}

// Interface terms of one pencil: the element is the "+" side of plane e_d
// (its first node receives -(s/w) F*) and the "-" side of plane e_d + 1 (its
// last node receives +(s/w) F*); fn is the pencil's node index on those faces.
// INIT: the terms are the accumulators' initial value (FP64: they are then
// loaded long before their first use), else they are added at the end (mixed:
// after the element's reference geopotential is restored in the pair sums).
template <bool INIT, int N, typename R>
__device__ __forceinline__ void face_lift(const EsdgGrid& g, const EsdgVolArgs& a, int e, int d,
                                          int fn, R (&acc)[N + 1][5]) {
  constexpr int NPEN = (N + 1) * (N + 1);
  // element indices selected without dynamic array indexing (no local memory)
  const int i0 = e % g.K[0], i1 = (e / g.K[0]) % g.K[1], i2 = e / (g.K[0] * g.K[1]);
  const int Pm = (d == 0) ? i0 : ((d == 1) ? i1 : i2);
  const int ia = (d == 0) ? i1 : i0;  // index along esdg_others(d).o1
  const int ib = (d == 2) ? i1 : i2;  // index along esdg_others(d).o2
  const int Kd = (d == 0) ? g.K[0] : ((d == 1) ? g.K[1] : g.K[2]);
  const int per = (d == 0) ? g.periodic[0] : ((d == 1) ? g.periodic[1] : g.periodic[2]);
  int Pp = Pm + 1;
  if (Pp == Kd && per) Pp = 0;
  const long long fm = esdg_face_id(g, d, Pm, ia, ib);
  const long long fp = esdg_face_id(g, d, Pp, ia, ib);
  const R* ff = reinterpret_cast<const R*>(a.fflux);
#pragma unroll
  for (int v = 0; v < 5; v++) {
    const R m = ff[((size_t)fm * 5 + v) * NPEN + fn], p = ff[((size_t)fp * 5 + v) * NPEN + fn];
    if (INIT) {
      acc[0][v] = -m;
      acc[N][v] = p;
    } else {
      acc[0][v] -= m;
      acc[N][v] += p;
    }
  }
}

// FP64 node primitives from the conserved state: rho/4, b/2 = rho/(4p),
// 1/b = 2p/rho, u/2 and phi/2, with p = (gamma - 1)(E - rho phi - |rho u|^2/(2 rho)).
// Power-of-two factors are applied exactly on the exponent field and b/2 is
// taken as 1/(2 (1/b)): 15 FP64-pipe instructions per node.
template <int NP>
__device__ __forceinline__ void prims64(double q0, double q1, double q2, double q3, double q4,
                                        double phi, double gm1, double* S, int n) {
  const double ir = esdg_rcp(q0);
  const double hi = esdg_ldexp(ir, -1);  // 1/(2 rho)
  const double u0 = q1 * hi, u1 = q2 * hi, u2 = q3 * hi;
  double ei = fma(-q0, phi, q4);
  ei = fma(-q1, u0, ei);
  ei = fma(-q2, u1, ei);
  ei = fma(-q3, u2, ei);
  const double p = gm1 * ei;
  const double ib = esdg_ldexp(p, 1) * ir;  // 1/b = 2p/rho
  S[0 * NP + n] = esdg_ldexp(q0, -2);
  S[1 * NP + n] = esdg_ldexp(esdg_rcp(ib), -1);
  S[2 * NP + n] = ib;
  S[3 * NP + n] = u0;
  S[4 * NP + n] = u1;
  S[5 * NP + n] = u2;
  S[6 * NP + n] = esdg_ldexp(phi, -1);
}

// Does any pair of this element leave the FP64 series range?  All
// |x_n/x_0 - 1| below 0.0095 (x = rho, b) bound |f| < 0.0096 for every pair,
// i.e. u < 1e-4.  Integer-repacked FP32 comparisons keep the FP64 pipe free.
template <int NP>
__device__ __forceinline__ bool out_of_series64(const double* S, int n) {
  const float r0 = esdg_d2f(S[0]), rn = esdg_d2f(S[n]);
  const float b0 = esdg_d2f(S[NP]), bn = esdg_d2f(S[NP + n]);
  return fabsf(rn - r0) > 0.0095f * r0 || fabsf(bn - b0) > 0.0095f * b0;
}

// Mixed-precision node prologue: FP32 primitives, the pressure recovered in
// FP64 (E - rho phi cancels there) and, with a background, the FP64
// perturbations rho' = rho - rho_bg and p' = p - p_bg rounded to FP32; the
// perturbation of b = rho/(2p) follows exactly from them,
//   b - b_bg = (rho' p_bg - rho_bg p') / (2 p p_bg),
// evaluated in FP32 (its rounding is relative to the perturbations).  phh is
// the geopotential relative to the element's first node, halved (FP32
// geometry).  5 FP64 instructions per node with a background.
template <int NP, bool BG>
__device__ __forceinline__ void prims32(double q0, double q1, double q2, double q3, double q4,
                                        double phi, float phh, double gm1, float* S, int n,
                                        double rb = 0.0, double bb = 0.0, double pbg = 0.0,
                                        float* Bf = nullptr) {
  const float q0f = esdg_d2f(q0), q1f = esdg_d2f(q1), q2f = esdg_d2f(q2), q3f = esdg_d2f(q3);
  const float irf = esdg_rcpf(q0f);
  const float hf = 0.5f * irf;
  const float u0 = q1f * hf, u1 = q2f * hf, u2 = q3f * hf;
  const float ke = fmaf(q3f, u2, fmaf(q2f, u1, q1f * u0));
  const double p = gm1 * (fma(-q0, phi, q4) - esdg_f2d(ke));
  const float pf = esdg_d2f(p);
  const float rq = 0.25f * q0f;
  S[0 * NP + n] = rq;
  S[1 * NP + n] = rq * esdg_rcpf(pf);
  S[2 * NP + n] = 2.0f * pf * irf;
  S[3 * NP + n] = u0;
  S[4 * NP + n] = u1;
  S[5 * NP + n] = u2;
  S[6 * NP + n] = phh;
  if constexpr (BG) {
    const float rpf = esdg_d2f(q0 - rb), ppf = esdg_d2f(p - pbg);
    const float rbf = esdg_d2f(rb), bbf = esdg_d2f(bb), pbf = esdg_d2f(pbg);
    Bf[0 * NP + n] = 0.25f * rpf;
    Bf[1 * NP + n] = 0.25f * fmaf(rpf, pbf, -rbf * ppf) * esdg_rcpf(pf * pbf);  // b'/2
    Bf[2 * NP + n] = 0.25f * rbf;
    Bf[3 * NP + n] = 0.5f * bbf;
    Bf[4 * NP + n] = esdg_rcpf(bbf);
    Bf[5 * NP + n] = pbf;
    Bf[6 * NP + n] = ppf;
  }
}

// Mixed-precision stage update of one node: r = -(1/J) (volume + lifts) in
// FP32, plus the background's right-hand side and the Coriolis source, all in
// FP32 (they join an FP32 increment); FP64 only in q += B dq.  Arrays are per
// node with stride NP between variables: rbg (3, background rhs), qin (5),
// dqold (5) may be in shared or global memory; dq and qio are the node's
// global locations.
template <int NP, bool BG>
__device__ __forceinline__ void stage32(float (&r)[5], const double* rbg, const EsdgPhys& P,
                                        double y, const double* qin, const float* dqold, float* dq,
                                        double* qio, double rkA, double rkB, double dt) {
  if constexpr (BG) {
    r[1] += esdg_d2f(rbg[0]);
    r[2] += esdg_d2f(rbg[NP]);
    r[3] += esdg_d2f(rbg[2 * NP]);
  }
  if ((P.f0 != 0.0) || (P.beta != 0.0)) {
    const float f = esdg_d2f(P.f0 + P.beta * (y - P.y0));
    r[1] = fmaf(f, esdg_d2f(qin[2 * NP]), r[1]);
    r[2] = fmaf(-f, esdg_d2f(qin[NP]), r[2]);
  }
  const float A = esdg_d2f(rkA), B = esdg_d2f(rkB), dtf = esdg_d2f(dt);
#pragma unroll
  for (int v = 0; v < 5; v++) {
    const float dv = fmaf(A, dqold[(size_t)v * NP], dtf * r[v]);
    dq[(size_t)v * NP] = dv;
    qio[(size_t)v * NP] = qin[(size_t)v * NP] + esdg_f2d(B * dv);
  }
}

// One tile: elements e0 .. e0 + EPB - 1 of one mesh, processed by a CTA of
// SH::THREADS threads with SH::SMEM bytes of shared memory at smraw.
template <int N, bool MIXED, int MODE, bool BG, int EPB_ = 0>
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
        if constexpr (BG) {
          const double* bge = a.bg + (size_t)e * 3 * NP;
          prims32<NP, true>(q0, q1, q2, q3, q4, phi, phh, gm1, S, n, bge[n], bge[NP + n],
                            bge[2 * NP + n], S + SH::F_BG * NP);
        } else {
          prims32<NP, false>(q0, q1, q2, q3, q4, phi, phh, gm1, S, n);
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
      const R phi0 = esdg_d2f(a.vgeo64[((size_t)e * ESDG_NVGEO + 10) * NP]);
#pragma unroll
      for (int i = 0; i < Nq; i++) acc[i][4] = fmaf(phi0, acc[i][0], acc[i][4]);
      face_lift<false, N, R>(g, a, e, d, s + Nq * t, acc);
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
      stage32<NP, BG>(r32, BG ? a.rhs_bg + (size_t)e2 * 3 * NP + n : nullptr, P, y, a.q_in + qb,
                      dq + qb, dq + qb, a.q_io + qb, a.rkA, a.rkB, a.dt);
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
    if constexpr (BG) {  // the background's own FP64 momentum right-hand side
      r[1] += a.rhs_bg[((size_t)e2 * 3 + 0) * NP + n];
      r[2] += a.rhs_bg[((size_t)e2 * 3 + 1) * NP + n];
      r[3] += a.rhs_bg[((size_t)e2 * 3 + 2) * NP + n];
    }
    if (rotating) {
      const double y = a.x[((size_t)e2 * 3 + 1) * NP + n];
      double f = P.f0 + P.beta * (y - P.y0);
      if constexpr (DT_IN_R) f *= a.dt;
      r[1] = fma(f, a.q_in[qb + 2 * NP], r[1]);
      r[2] = fma(-f, a.q_in[qb + NP], r[2]);
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
          const double dv = fma(a.rkA, dq[qb + (size_t)v * NP], r[v]);
          dq[qb + (size_t)v * NP] = dv;
          a.q_io[qb + (size_t)v * NP] = fma(a.rkB, dv, a.q_in[qb + (size_t)v * NP]);
        }
      }
    }
  }
}

template <int N, bool MIXED, int MODE, bool BG>
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
// dynamic shared memory a pipelined tile may use (227 KB less static use)
#define ESDG_PIPE_SMEM_MAX (232448 - 1024)

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
  using SH = Shape<N, false, false>;
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
  const unsigned long long src = reinterpret_cast<unsigned long long>(c.src);
  const unsigned long long end = src + (unsigned long long)c.n * c.esz;
  const unsigned long long lim = reinterpret_cast<unsigned long long>(c.lim);
  BlockSpan s;
  s.a = src & ~15ull;
  s.sh = (int)((src - s.a) / (unsigned)c.esz);
  const unsigned long long up = (end + 15ull) & ~15ull;
  s.b = up <= lim ? up : (end & ~15ull);
  if (s.b < s.a) s.b = s.a;
  s.tail0 = s.b >= end ? c.n : (s.b > src ? (int)((s.b - src) / (unsigned)c.esz) : 0);
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
template <typename ISS, int MAXB>
__device__ __forceinline__ void pipe_issue(int tid, const BlockCopy (&bl)[MAXB], int nb,
                                           unsigned long long* bar, unsigned extra = 0,
                                           const void* xsrc = nullptr, void* xdst = nullptr,
                                           unsigned phantom = 0) {
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
}

template <int N, int MODE, bool TABLE>
__global__ void __launch_bounds__(Shape<N, false, false>::THREADS, 1)
    k_volume_pipe64(const EsdgMember one, const EsdgMember* __restrict__ members,
                    const int2* __restrict__ tiles, const int* __restrict__ ntiles_d, int ntiles_1,
                    EsdgLGL L, double rkA, double rkB, unsigned phantom, int t1, int s1) {
  static_assert(!TABLE || MODE == 1, "the batched kernel applies an RK stage");
  using SH = Shape<N, false, false>;
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
          X[5 * NP + n] = gr[9 * NP + n];
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
        if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
        return;
      }
    } else {
      __syncthreads();
    }

    // ---- epilogue: one thread per node --------------------------------------
    const double* D0 = sm + PP::DQ + esdg_block_shift(reinterpret_cast<const double*>(a.dq) + (size_t)e0 * 5 * NP);
    // descriptor fields in registers (the stores below would force reloads)
    const double dt = a.dt;
    const EsdgPhys Pl = P;
    const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
    const double* xg = a.x;
    double* const dqp = reinterpret_cast<double*>(a.dq);
    double* const qio = a.q_io;
    double* const rhsp = a.rhs;
    for (int idx = tid; idx < EPB * NP; idx += T) {
      const int el2 = idx / NP, n = idx - el2 * NP, e2 = e0 + el2;
      if (el2 >= ne) continue;
      const double* S = sm + PP::S0 + (size_t)el2 * NF * NP;
      const double* X = sm + PP::EPI + (size_t)el2 * 6 * NP;
      double iJ = X[5 * NP + n];
      if constexpr (MODE != 0) iJ *= dt;
      double r[5];
#pragma unroll
      for (int v = 0; v < 5; v++) r[v] = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
      if (rot) {
        const double y = xg[((size_t)e2 * 3 + 1) * NP + n];
        double f = Pl.f0 + Pl.beta * (y - Pl.y0);
        if constexpr (MODE != 0) f *= dt;
        r[1] = fma(f, X[2 * NP + n], r[1]);
        r[2] = fma(-f, X[NP + n], r[2]);
      }
      const size_t qb = (size_t)e2 * 5 * NP + n;
      if constexpr (MODE == 0) {
#pragma unroll
        for (int v = 0; v < 5; v++) rhsp[qb + (size_t)v * NP] = r[v];
      } else {
        const double* D = D0 + (size_t)el2 * 5 * NP;
#pragma unroll
        for (int v = 0; v < 5; v++) {
          const double dv = fma(rkA, D[v * NP + n], r[v]);
          dqp[qb + (size_t)v * NP] = dv;
          qio[qb + (size_t)v * NP] = fma(rkB, dv, X[v * NP + n]);
        }
      }
    }
  }
}

// ---- pipelined persistent mixed-precision kernel (with a background) ------
template <int N, int MODE>
struct Pipe32 {
  using SH = Shape<N, true, true>;
  static constexpr int NP = SH::NP, EPB = SH::EPB, P = NP * EPB;
  static constexpr int up16(int b) { return (b + 15) & ~15; }
  static constexpr int PHS = (NP + 4) & ~1;  // even per-element stride: every target 16-byte aligned
  // byte offsets, 16-byte aligned; copy targets hold 32 extra bytes (the
  // aligned span around each block)
  static constexpr int RAW_Q = 0;                                  // [el][5][NP]  double
  static constexpr int RAW_PHI = up16(RAW_Q + 8 * (5 * P + 4));    // [el][PHS]    double
  static constexpr int RAW_BG = up16(RAW_PHI + 8 * EPB * PHS);     // [el][3][NP]  double
  static constexpr int RAW_G = up16(RAW_BG + 8 * (3 * P + 4));     // [el][11][NP] float
  static constexpr int S0 = up16(RAW_G + 4 * (ESDG_NVGEO * P + 8));  // [el][NF][NP] float
  static constexpr int EPI_Q = up16(S0 + 4 * SH::NF * P);         // [el][5][NP]  double
  static constexpr int EPI_J = up16(EPI_Q + 8 * 5 * P);           // [el][NP]     float
  static constexpr int CUR_RB = up16(EPI_J + 4 * P);              // [el][3][NP]  double
  static constexpr int CUR_DQ = up16(CUR_RB + 8 * (3 * P + 4));   // [el][5][NP]  float
  static constexpr int TOTAL = MODE ? up16(CUR_DQ + 4 * (5 * P + 8)) : CUR_DQ;
  static constexpr size_t SMEM = (size_t)TOTAL;
};

template <int N, int MODE, bool TABLE>
__global__ void __launch_bounds__(Shape<N, true, true>::THREADS, 1)
    k_volume_pipe32(const EsdgMember one, const EsdgMember* __restrict__ members,
                    const int2* __restrict__ tiles, const int* __restrict__ ntiles_d, int ntiles_1,
                    EsdgLGL L, double rkA, double rkB, unsigned phantom, int t1, int s1) {
  static_assert(!TABLE || MODE == 1, "the batched kernel applies an RK stage");
  using SH = Shape<N, true, true>;
  using PP = Pipe32<N, MODE>;
  constexpr int Nq = SH::Nq, NP = SH::NP, NPEN = SH::NPEN, EPB = SH::EPB, NF = SH::NF;
  constexpr int T = SH::THREADS;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ __align__(16) PipeCtl<TABLE> ctl;
  __shared__ float phi0s[EPB];  // each element's reference geopotential
  double* const rawq = reinterpret_cast<double*>(smraw + PP::RAW_Q);
  double* const rawphi = reinterpret_cast<double*>(smraw + PP::RAW_PHI);
  double* const rawbg = reinterpret_cast<double*>(smraw + PP::RAW_BG);
  float* const rawg = reinterpret_cast<float*>(smraw + PP::RAW_G);
  float* const sm = reinterpret_cast<float*>(smraw + PP::S0);
  double* const epq = reinterpret_cast<double*>(smraw + PP::EPI_Q);
  float* const epj = reinterpret_cast<float*>(smraw + PP::EPI_J);
  double* const currb = reinterpret_cast<double*>(smraw + PP::CUR_RB);
  float* const curdq = reinterpret_cast<float*>(smraw + PP::CUR_DQ);
  const int tid = threadIdx.x;
  const int ntiles = TABLE ? *ntiles_d : ntiles_1;

  auto phi_src = [](const EsdgMember* M, int e) {
    return M->a.vgeo64 + ((size_t)e * ESDG_NVGEO + 10) * NP;
  };
  using ISS = Issuers<T, SH::PENCILS>;
  struct Next {
    int4 tr;  // (member, first element, elements)
    int E;
    const double* q;
    const double* bg;
    const float* vg;
    const double* v64;
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
    x.vg = reinterpret_cast<const float*>(x.Mg->a.vgeo);
    x.v64 = x.Mg->a.vgeo64;
    return x;
  };
  // issuing lanes: the next tile's (member, e0), descriptor and RAW blocks into slot s
  auto issue_next = [&](const Next& x, int s, unsigned ph = 0) {
    if (tid == ISS::FIRST) ctl.info[s] = x.tr;
    const int e0 = x.tr.y, ne = x.tr.z;
    const double* v64end = x.v64 + (size_t)x.E * ESDG_NVGEO * NP;
    BlockCopy bl[3 + EPB];
    bl[0] = {rawq, x.q + (size_t)e0 * 5 * NP, x.q + (size_t)x.E * 5 * NP, ne * 5 * NP, 8};
    bl[1] = {rawbg, x.bg + (size_t)e0 * 3 * NP, x.bg + (size_t)x.E * 3 * NP, ne * 3 * NP, 8};
    bl[2] = {rawg, x.vg + (size_t)e0 * ESDG_NVGEO * NP, x.vg + (size_t)x.E * ESDG_NVGEO * NP,
             ne * ESDG_NVGEO * NP, 4};
#pragma unroll
    for (int el = 0; el < EPB; el++)
      bl[3 + el] = {rawphi + (size_t)el * PP::PHS, x.v64 + ((size_t)(e0 + el) * ESDG_NVGEO + 10) * NP,
                    v64end, el < ne ? NP : 0, 8};
    if constexpr (TABLE)
      pipe_issue<ISS>(tid, bl, 3 + EPB, &ctl.bars[0], (unsigned)sizeof(EsdgMember), x.Mg, &ctl.desc[s], ph);
    else
      pipe_issue<ISS>(tid, bl, 3 + EPB, &ctl.bars[0], 0, nullptr, nullptr, ph);
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
          {currb, a.rhs_bg + (size_t)e0 * 3 * NP, a.rhs_bg + (size_t)E * 3 * NP, ne * 3 * NP, 8},
          {curdq, dqg + (size_t)e0 * 5 * NP, dqg + (size_t)E * 5 * NP, MODE ? ne * 5 * NP : 0, 4}};
      pipe_issue<ISS>(tid, cb, 2, &ctl.bars[1]);
      if (TABLE && next < ntiles) nx = fetch(next);  // global loads: early
    }
    // ---- prologue (descriptor fields held in registers: the shared-memory
    // stores below would otherwise force their reloads) -----------------------
    {
      const double gm1 = P.gamma - 1.0;
      const float* vg = reinterpret_cast<const float*>(a.vgeo);
      const double* v64 = a.vgeo64;
      const double* qr0 = rawq + esdg_block_shift(a.q_in + (size_t)e0 * 5 * NP);
      const double* br0 = rawbg + esdg_block_shift(a.bg + (size_t)e0 * 3 * NP);
      const float* gr0 = rawg + esdg_block_shift(vg + (size_t)e0 * ESDG_NVGEO * NP);
      for (int idx = tid; idx < EPB * NP; idx += T) {
        const int el2 = idx / NP, n = idx - el2 * NP;
        float* S = sm + (size_t)el2 * NF * NP;
        if (el2 < ne) {
          const double* qr = qr0 + (size_t)el2 * 5 * NP;
          const double* br = br0 + (size_t)el2 * 3 * NP;
          const float* gr = gr0 + (size_t)el2 * ESDG_NVGEO * NP;
          const double* phr = rawphi + (size_t)el2 * PP::PHS +
                              esdg_block_shift(v64 + ((size_t)(e0 + el2) * ESDG_NVGEO + 10) * NP);
          const double q0 = qr[n], q1 = qr[NP + n], q2 = qr[2 * NP + n], q3 = qr[3 * NP + n],
                       q4 = qr[4 * NP + n];
          prims32<NP, true>(q0, q1, q2, q3, q4, phr[n], gr[10 * NP + n], gm1, S, n, br[n],
                            br[NP + n], br[2 * NP + n], S + SH::F_BG * NP);
          if (n == 0) phi0s[el2] = esdg_d2f(phr[0]);
#pragma unroll
          for (int k = 0; k < 9; k++) S[(SH::F_NH + k) * NP + n] = gr[k * NP + n];
          double* X = epq + (size_t)el2 * 5 * NP;
          X[n] = q0;
          X[NP + n] = q1;
          X[2 * NP + n] = q2;
          X[3 * NP + n] = q3;
          X[4 * NP + n] = q4;
          epj[(size_t)el2 * NP + n] = gr[9 * NP + n];
        } else {  // padding element: any valid state, results are discarded
          S[0 * NP + n] = 0.25f;
          S[1 * NP + n] = 0.5f;
          S[2 * NP + n] = 1.0f;
          for (int k = 3; k < NF; k++) S[k * NP + n] = 0.0f;
        }
      }
    }
    __syncthreads();  // RAW consumed

    int need_logs = 0;
    for (int idx = tid; idx < EPB * NP; idx += T) {
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
      const float* S = sm + (size_t)el * NF * NP;
      const float ce = esdg_d2f(0.5 * P.igm1);
      if (need_logs)
        pencil_pass<N, true, true, true>(S, d, base, stride, L, ce, acc);
      else
        pencil_pass<N, true, false, true>(S, d, base, stride, L, ce, acc);
      const float phi0 = phi0s[el];
#pragma unroll
      for (int i = 0; i < Nq; i++) acc[i][4] = fmaf(phi0, acc[i][0], acc[i][4]);
      face_lift<false, N, float>(g, a, e, d, ps + Nq * pt, acc);
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
      if (tid == 0) atomicExch(&g_esdg_vol_timeout, 1);
      return;
    }

    // ---- epilogue: one thread per node ----------------------------------------
    const double* RB0 = currb + esdg_block_shift(a.rhs_bg + (size_t)e0 * 3 * NP);
    const float* D0 = curdq + esdg_block_shift(reinterpret_cast<const float*>(a.dq) + (size_t)e0 * 5 * NP);
    const EsdgPhys Pl = P;
    const bool rot = (Pl.f0 != 0.0) || (Pl.beta != 0.0);
    const double* xg = a.x;
    float* const dqp = reinterpret_cast<float*>(a.dq);
    double* const qio = a.q_io;
    double* const rhsp = a.rhs;
    const double dtv = a.dt;
    for (int idx = tid; idx < EPB * NP; idx += T) {
      const int el2 = idx / NP, n = idx - el2 * NP, e2 = e0 + el2;
      if (el2 >= ne) continue;
      const float* S = sm + (size_t)el2 * NF * NP;
      const double* X = epq + (size_t)el2 * 5 * NP;
      const float iJ = epj[(size_t)el2 * NP + n];
      const double* RB = RB0 + (size_t)el2 * 3 * NP;
      const size_t qb = (size_t)e2 * 5 * NP + n;
      if constexpr (MODE != 0) {
        float r32[5];
#pragma unroll
        for (int v = 0; v < 5; v++)
          r32[v] = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
        const double y = rot ? xg[((size_t)e2 * 3 + 1) * NP + n] : 0.0;
        stage32<NP, true>(r32, RB + n, Pl, y, X + n, D0 + (size_t)el2 * 5 * NP + n, dqp + qb,
                          qio + qb, rkA, rkB, dtv);
      } else {  // right-hand side in FP64
        double r[5];
#pragma unroll
        for (int v = 0; v < 5; v++) {
          const float rv = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
          r[v] = esdg_f2d(rv);
        }
        r[1] += RB[n];
        r[2] += RB[NP + n];
        r[3] += RB[2 * NP + n];
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
  using SH = Shape<N, false, false>;
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
  using SH = Shape<N, true, true>;
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
  using SH = Shape<N, MIXED, MIXED>;
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

template <int N, bool MIXED, int MODE, bool BG>
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
      if (a.bg) {                                                              \
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
