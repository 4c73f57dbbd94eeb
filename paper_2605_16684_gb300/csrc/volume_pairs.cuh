// volume_pairs.cuh -- the arithmetic of the flux-differencing volume kernels
// (Section 3, Eq. (nm:semi); Section 4.1): tile shapes, node data, the two-point
// pair in FP64 and FP32 (with and without a hydrostatic background), the pencil
// pass, the interface lifts, the node prologues and the mixed stage update.
// Shared by the per-tile kernels (volume_tile.cuh) and the pipelined
// persistent kernels (volume_pipe.cuh), so both give bitwise the same results.
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

// BG: 0 no background, 1 a background at rest (hydrostatic), 2 a moving
// background (one that carries a flow; mixed mode only)
template <int N, bool MIXED, int BG = 0, int EPB_ = 0>
struct Shape {
  static constexpr int Nq = N + 1, NP = Nq * Nq * Nq, NPEN = Nq * Nq;
  static constexpr int EPB = EPB_ > 0 ? EPB_ : Cfg<N, MIXED>::EPB;  // elements per CTA (tile)
  static constexpr int PENCILS = 3 * NPEN * EPB;
  static constexpr int THREADS = ((PENCILS + 31) / 32) * 32;
  // node fields: rq=rho/4, bh=b/2, ib=1/b, uh=u/2 (3), ph=phi/2, [lr, lb], nh=Ja/2 (9),
  // [background: rq'=rho'/4, bh'=b'/2, rq_bg, bh_bg, 1/b_bg, p_bg, p'=p-p_bg,
  //  moving background: u'/2 = (u - u_bg)/2 (3)]
  static constexpr int F_LR = 7, F_LB = 8;
  static constexpr int F_NH = MIXED ? 7 : 9;
  static constexpr int F_BG = F_NH + 9;
  static constexpr int NF = F_NH + 9 + (BG ? 7 : 0) + (BG == 2 ? 3 : 0);
  using R = typename std::conditional<MIXED, float, double>::type;
  static constexpr size_t SMEM = sizeof(R) * (size_t)NF * NP * EPB;
};

template <typename R>
struct Node {
  R rq, bh, ib, u0, u1, u2, ph, n0, n1, n2, lr, lb;
  R rqp, bhp, rqb, bhb, ibb, pb, pp;  // perturbation and background (mixed mode with a background)
  R up0, up1, up2;                    // u'/2 (a moving background)
};

template <typename R, bool LOGS, int F_NH, int NP, int BG = 0>
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
  if (BG == 2) {
    const R* b = S + (F_NH + 16) * NP;
    a.up0 = b[0 * NP + n];
    a.up1 = b[1 * NP + n];
    a.up2 = b[2 * NP + n];
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

// Log branch of a log-mean difference relative to a background, for field
// values x = x_bg + x' at the pair's nodes A, B (the density's quarter or b's
// half: the mean is 4 d/L, 1/<b>_log is L/(2 d)).  With d = x_A - x_B =
// d_bg + d', L = ln(x_A/x_B) = L_bg + l and l = log1p(x'_A/x_bg,A) -
// log1p(x'_B/x_bg,B):
//   d/L - d_bg/L_bg = (d' L_bg - d_bg l) / (L_bg (L_bg + l)),
//   L/d - L_bg/d_bg = (l d_bg - L_bg d') / (d_bg d),
// each term carrying a perturbation factor, where the plain difference of the
// two means would round relative to the means themselves (a strongly
// stratified background, e.g. a scale height of a few kilometres across one
// element, takes every vertical pair to the log branch).  Needs L_bg and d_bg
// away from zero (the background's own u at or above the series threshold).
struct LogDiff {
  float L, l;  // L_bg, l
};
__device__ __forceinline__ LogDiff esdg_logdiff(float xa, float xb, float pa, float pb) {
  return LogDiff{log1pf((xa - xb) * esdg_rcpf(xb)),
                 log1pf(pa * esdg_rcpf(xa)) - log1pf(pb * esdg_rcpf(xb))};
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
    if (urb < ESDG_LOG_EPS32 || ur < ESDG_LOG_EPS32) {
      // a near-uniform background or a perturbation that cancels its ratio: the
      // plain difference is relative to the perturbation already
      const float rlogb = (urb < ESDG_LOG_EPS32) ? srb * esdg_Q2f(urb)
                                                 : (4.0f * drb) / log1pf(drb * esdg_rcpf(B.rqb));
      rlogp = rlog - rlogb;
    } else {
      const LogDiff g = esdg_logdiff(A.rqb, B.rqb, A.rqp, B.rqp);
      rlogp = 4.0f * fmaf(A.rqp - B.rqp, g.L, -drb * g.l) / (g.L * (g.L + g.l));
    }
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

// The FP32 pair relative to a moving background (u_bg != 0, e.g. a balanced
// jet, whose convective fluxes are far larger than their divergence): every
// flux is formed as H - H_bg.  With primes for state minus background, sums
// over the pair of the halved node fields ({{u}} = u_i/2 + u_l/2) and
// un = {{u}}.n, un' = {{u'}}.n:
//   Fr - Fr_bg = (<rho>_log - <rho_bg>_log) un + <rho_bg>_log un',
//   M - M_bg   = (Fr - Fr_bg) {{u}} + Fr_bg {{u'}} + (p* - p*_bg) n,
//   FE - FE_bg = (Fr - Fr_bg) W + Fr_bg W' + (p* - p*_bg) un + p*_bg un',
// Fr_bg = <rho_bg>_log {{u_bg}}.n, W = ce/<b>_log + u_i.u_l/2 + {{phi}} and
// W' = ce (1/<b>_log - 1/<b_bg>_log) + (u'_i.u_l + u_bg,i.u'_l)/2.  Both
// log-mean differences come from divided differences of their series (the
// density's as in pair32bg; 1/<b>_log = A(u_b)/{{b}} with A(u) = 1 + u/3 +
// u^2/5 + u^3/7, so its difference is A(u_b)(1/{{b}} - 1/{{b_bg}}) +
// (A(u_b) - A(u_b,bg))/{{b_bg}}), so every term carries a perturbation
// factor.  The pressure mean and the gravity parts are those of pair32bg.
template <bool LOGS>
__device__ __forceinline__ void pair32bgm(const Node<float>& A, const Node<float>& B, float dil,
                                          float dli, float ce, float* ai, float* al) {
  const float sr = A.rq + B.rq;
  const float sb = A.bh + B.bh;
  const float rsb = esdg_rcpf(sb);
  const float pt = sr * rsb;
  const float dr = A.rq - B.rq, db = A.bh - B.bh;
  const float rsr = esdg_rcpf(sr);
  const float fr = dr * rsr, ur = fr * fr;
  const float fb = db * rsb, ub = fb * fb;
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
  const float drb = A.rqb - B.rqb, dbb = A.bhb - B.bhb;
  const float rsrb = esdg_rcpf(srb), rsbb = esdg_rcpf(sbb);
  const float frb = drb * rsrb, urb = frb * frb;
  const float fbb = dbb * rsbb, ubb = fbb * fbb;
  float rlog, iblog, rlogp, iblogp;
  if (!LOGS || (ur < ESDG_LOG_EPS32 && ub < ESDG_LOG_EPS32 && urb < ESDG_LOG_EPS32 &&
                ubb < ESDG_LOG_EPS32)) {
    const float q2 = esdg_Q2f(ur);
    rlog = sr * q2;
    const float ab = esdg_Af(ub);
    iblog = rsb * ab;
    const float fdiff = 2.0f * (A.rqp * B.rqb - B.rqp * A.rqb) * rsr * rsrb;
    const float udiff = fdiff * (fr + frb);
    const float s2 = fmaf(-88.0f / 945.0f, fmaf(ur, ur, fmaf(ur, urb, urb * urb)),
                          fmaf(-8.0f / 45.0f, ur + urb, -2.0f / 3.0f));
    rlogp = fmaf(srp, q2, srb * udiff * s2);
    const float sbp = A.bhp + B.bhp;
    const float gdiff = 2.0f * (A.bhp * B.bhb - B.bhp * A.bhb) * rsb * rsbb;
    const float vdiff = gdiff * (fb + fbb);
    // divided difference of A(u) = 1 + u/3 + u^2/5 + u^3/7
    const float sa = fmaf(1.0f / 7.0f, fmaf(ub, ub, fmaf(ub, ubb, ubb * ubb)),
                          fmaf(0.2f, ub + ubb, 1.0f / 3.0f));
    iblogp = fmaf(-ab * sbp, rsb * rsbb, rsbb * vdiff * sa);
  } else {
    rlog = (ur < ESDG_LOG_EPS32) ? sr * esdg_Q2f(ur)
                                 : (4.0f * dr) / log1pf(dr * esdg_rcpf(B.rq));
    iblog = (ub < ESDG_LOG_EPS32) ? rsb * esdg_Af(ub)
                                  : log1pf(db * esdg_rcpf(B.bh)) / (2.0f * db);
    if (urb < ESDG_LOG_EPS32 || ur < ESDG_LOG_EPS32) {
      const float rlogb = (urb < ESDG_LOG_EPS32) ? srb * esdg_Q2f(urb)
                                                 : (4.0f * drb) / log1pf(drb * esdg_rcpf(B.rqb));
      rlogp = rlog - rlogb;
    } else {
      const LogDiff g = esdg_logdiff(A.rqb, B.rqb, A.rqp, B.rqp);
      rlogp = 4.0f * fmaf(A.rqp - B.rqp, g.L, -drb * g.l) / (g.L * (g.L + g.l));
    }
    if (ubb < ESDG_LOG_EPS32 || ub < ESDG_LOG_EPS32) {
      const float iblogb = (ubb < ESDG_LOG_EPS32) ? rsbb * esdg_Af(ubb)
                                                  : log1pf(dbb * esdg_rcpf(B.bhb)) / (2.0f * dbb);
      iblogp = iblog - iblogb;
    } else {
      const LogDiff g = esdg_logdiff(A.bhb, B.bhb, A.bhp, B.bhp);
      iblogp = fmaf(g.l, dbb, -g.L * (A.bhp - B.bhp)) / (2.0f * dbb * db);
    }
  }
  const float rlogb = rlog - rlogp;
  const float n0 = A.n0 + B.n0, n1 = A.n1 + B.n1, n2 = A.n2 + B.n2;
  const float u0 = A.u0 + B.u0, u1 = A.u1 + B.u1, u2 = A.u2 + B.u2;
  const float v0 = A.up0 + B.up0, v1 = A.up1 + B.up1, v2 = A.up2 + B.up2;  // {{u'}}
  const float un = fmaf(u2, n2, fmaf(u1, n1, u0 * n0));
  const float unp = fmaf(v2, n2, fmaf(v1, n1, v0 * n0));
  const float Frp = fmaf(rlogp, un, rlogb * unp);  // Fr - Fr_bg
  const float Frb = rlogb * (un - unp);            // Fr_bg
  const float m0 = fmaf(Frp, u0, fmaf(Frb, v0, ptp * n0));
  const float m1 = fmaf(Frp, u1, fmaf(Frb, v1, ptp * n1));
  const float m2 = fmaf(Frp, u2, fmaf(Frb, v2, ptp * n2));
  const float uu = fmaf(A.u2, B.u2, fmaf(A.u1, B.u1, A.u0 * B.u0));
  const float t = fmaf(2.0f, uu, A.ph + B.ph);
  // (u'_i.u_l + u_bg,i.u'_l)/2 from the halved fields, u_bg,i/2 = u_i/2 - u'_i/2
  const float c0 = A.u0 - A.up0, c1 = A.u1 - A.up1, c2 = A.u2 - A.up2;
  const float tp = 2.0f * fmaf(A.up2, B.u2, fmaf(A.up1, B.u1, fmaf(A.up0, B.u0,
                              fmaf(c2, B.up2, fmaf(c1, B.up1, c0 * B.up0)))));
  const float FE = fmaf(Frp, fmaf(iblog, ce, t),
                        fmaf(Frb, fmaf(iblogp, ce, tp), fmaf(ptp, un, (pt - ptp) * unp)));
  // gravity perturbation (as pair32bg)
  const float dph = B.ph - A.ph;
  const float dYi = 2.0f * (B.bhp * A.bhb - B.bhb * A.bhp) * A.ib * A.ibb;
  const float dYl = 2.0f * (A.bhp * B.bhb - A.bhb * B.bhp) * B.ib * B.ibb;
  const float gi = dph * fmaf(dYi, rlog, sbb * A.ibb * rlogp);
  const float gl = -dph * fmaf(dYl, rlog, sbb * B.ibb * rlogp);
  ai[0] = fmaf(dil, Frp, ai[0]);
  ai[1] = fmaf(dil, fmaf(gi, n0, m0), ai[1]);
  ai[2] = fmaf(dil, fmaf(gi, n1, m1), ai[2]);
  ai[3] = fmaf(dil, fmaf(gi, n2, m2), ai[3]);
  ai[4] = fmaf(dil, FE, ai[4]);
  al[0] = fmaf(dli, Frp, al[0]);
  al[1] = fmaf(dli, fmaf(gl, n0, m0), al[1]);
  al[2] = fmaf(dli, fmaf(gl, n1, m1), al[2]);
  al[3] = fmaf(dli, fmaf(gl, n2, m2), al[3]);
  al[4] = fmaf(dli, FE, al[4]);
}

// ce: 1/(2(gamma - 1)) as float (mixed) or as the scaled series (FP64)
template <int N, bool MIXED, bool LOGS, int BG, typename CE>
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
      if constexpr (MIXED && BG == 2)
        pair32bgm<LOGS>(A, B, L.Dtf[i][l], L.Dtf[l][i], ce, acc[i], acc[l]);
      else if constexpr (MIXED && BG)
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
template <typename R>
struct FaceTerms {
  R m[5], p[5];  // (s/w) F* of the pencil's lower and upper face
};
template <int N, typename R>
__device__ __forceinline__ FaceTerms<R> face_fetch(const EsdgGrid& g, const EsdgVolArgs& a, int e,
                                                   int d, int fn) {
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
  FaceTerms<R> t;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    t.m[v] = ff[((size_t)fm * 5 + v) * NPEN + fn];
    t.p[v] = ff[((size_t)fp * 5 + v) * NPEN + fn];
  }
  return t;
}
// Mixed path: the terms are added after the pair sums (once the element's
// reference geopotential is restored in them); fetched before the pair pass,
// their gathers' latency hides behind it.
template <int N, typename R>
__device__ __forceinline__ void face_add(const FaceTerms<R>& t, R (&acc)[N + 1][5]) {
#pragma unroll
  for (int v = 0; v < 5; v++) {
    acc[0][v] -= t.m[v];
    acc[N][v] += t.p[v];
  }
}
// INIT: the terms are the accumulators' initial value (FP64: they are then
// loaded long before their first use), else they are added at once.
template <bool INIT, int N, typename R>
__device__ __forceinline__ void face_lift(const EsdgGrid& g, const EsdgVolArgs& a, int e, int d,
                                          int fn, R (&acc)[N + 1][5]) {
  const FaceTerms<R> t = face_fetch<N, R>(g, a, e, d, fn);
  if (INIT) {
#pragma unroll
    for (int v = 0; v < 5; v++) {
      acc[0][v] = -t.m[v];
      acc[N][v] = t.p[v];
    }
  } else {
    face_add<N, R>(t, acc);
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

// Mixed-precision node prologue without a background: FP32 primitives, the
// pressure recovered in FP64 (E - rho phi cancels there).  phh is the
// geopotential relative to the element's first node, halved (FP32 geometry).
template <int NP>
__device__ __forceinline__ void prims32(double q0, double q1, double q2, double q3, double q4,
                                        double phi, float phh, double gm1, float* S, int n) {
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
}

// The node fields of the FP32 pair loop relative to a hydrostatic background
// (Shape field order): s[0..6] = rho/4, b/2, 1/b, u/2 (3), phi_rel/2 and
// bgf[0..6] = rho'/4, b'/2, rho_bg/4, b_bg/2, 1/b_bg, p_bg, p'.
struct Prim32 {
  float s[7], bgf[7];
};
// Inputs: the FP64 state, phi (FP64) and phh = (phi - phi_0)/2 (FP32), the
// background's rho_bg and E_bg = p_bg/(gamma-1) + rho_bg phi (FP64) and its
// FP32 fields rqb = rho_bg/4, bhb = b_bg/2, ibb = 1/b_bg, pbf = p_bg.  FP64
// only where the state cancels against the background, three instructions:
//   rho' = rho - rho_bg,  E' = E - E_bg,  e' = E' - phi rho',
// then in FP32 (rounding relative to the perturbations, or to FP32 accuracy
// of fields that need no more):  rho and rho u rounded once, u = (rho u)/rho,
// p' = (gamma - 1)(e' - |rho u|^2/(2 rho)), p = p_bg + p', b = rho/(2p) and
//   b - b_bg = (rho' p_bg - rho_bg p') / (2 p p_bg)
// (exact identity, its rounding relative to the perturbations).
__device__ __forceinline__ Prim32 prims32bg(double q0, double q1, double q2, double q3, double q4,
                                            double phi, float phh, float gm1f, double rb,
                                            double eb, float rqb, float bhb, float ibb,
                                            float pbf) {
  const double rp = q0 - rb;
  const double ep = fma(-phi, rp, q4 - eb);
  const float rpf = esdg_d2f(rp), epf = esdg_d2f(ep);
  const float q0f = esdg_d2f(q0), q1f = esdg_d2f(q1), q2f = esdg_d2f(q2), q3f = esdg_d2f(q3);
  const float irf = esdg_rcpf(q0f);
  const float hf = 0.5f * irf;
  const float u0 = q1f * hf, u1 = q2f * hf, u2 = q3f * hf;
  const float ke = fmaf(q3f, u2, fmaf(q2f, u1, q1f * u0));
  const float ppf = gm1f * (epf - ke);
  const float pf = pbf + ppf;
  const float rq = 0.25f * q0f;
  Prim32 o;
  o.s[0] = rq;
  o.s[1] = rq * esdg_rcpf(pf);
  o.s[2] = 2.0f * pf * irf;
  o.s[3] = u0;
  o.s[4] = u1;
  o.s[5] = u2;
  o.s[6] = phh;
  o.bgf[0] = 0.25f * rpf;
  o.bgf[1] = fmaf(rpf, pbf, -4.0f * rqb * ppf) * esdg_rcpf(4.0f * pf * pbf);  // b'/2
  o.bgf[2] = rqb;
  o.bgf[3] = bhb;
  o.bgf[4] = ibb;
  o.bgf[5] = pbf;
  o.bgf[6] = ppf;
  return o;
}

// The node fields relative to a moving background: those of prims32bg plus
// up[0..2] = u'/2, u' = u - u_bg.  FP64 where the state cancels against the
// background, six instructions: rho' = rho - rho_bg, m' = m - m_bg (3),
// E' = E - E_bg, e' = E' - phi rho' (E_bg the background's total energy,
// kinetic part included); then in FP32, each rounding relative to the
// perturbation:
//   u' = (m' - rho' u_bg)/rho,  u = u_bg + u',
//   p' = (gamma - 1)(e' - KE'),  KE' = (m'.u + rho_bg u_bg.u')/2
// (KE' = m.u/2 - m_bg.u_bg/2 exactly), p = p_bg + p', b' as in prims32bg.
struct Prim32m {
  float s[7], bgf[7], up[3];
};
__device__ __forceinline__ Prim32m prims32bgm(double q0, double q1, double q2, double q3,
                                              double q4, double phi, float phh, float gm1f,
                                              double rb, double mb0, double mb1, double mb2,
                                              double eb, float rqb, float bhb, float ibb,
                                              float pbf, float ub0, float ub1, float ub2) {
  const double rp = q0 - rb;
  const double mp0 = q1 - mb0, mp1 = q2 - mb1, mp2 = q3 - mb2;
  const double ep = fma(-phi, rp, q4 - eb);
  const float rpf = esdg_d2f(rp), epf = esdg_d2f(ep);
  const float m0 = esdg_d2f(mp0), m1 = esdg_d2f(mp1), m2 = esdg_d2f(mp2);
  const float q0f = esdg_d2f(q0);
  const float irf = esdg_rcpf(q0f);
  const float v0 = fmaf(-rpf, ub0, m0) * irf, v1 = fmaf(-rpf, ub1, m1) * irf,
              v2 = fmaf(-rpf, ub2, m2) * irf;  // u'
  const float u0 = ub0 + v0, u1 = ub1 + v1, u2 = ub2 + v2;
  const float kb = (4.0f * rqb) * fmaf(ub2, v2, fmaf(ub1, v1, ub0 * v0));
  const float kep = 0.5f * fmaf(m2, u2, fmaf(m1, u1, fmaf(m0, u0, kb)));
  const float ppf = gm1f * (epf - kep);
  const float pf = pbf + ppf;
  const float rq = 0.25f * q0f;
  Prim32m o;
  o.s[0] = rq;
  o.s[1] = rq * esdg_rcpf(pf);
  o.s[2] = 2.0f * pf * irf;
  o.s[3] = 0.5f * u0;
  o.s[4] = 0.5f * u1;
  o.s[5] = 0.5f * u2;
  o.s[6] = phh;
  o.bgf[0] = 0.25f * rpf;
  o.bgf[1] = fmaf(rpf, pbf, -4.0f * rqb * ppf) * esdg_rcpf(4.0f * pf * pbf);  // b'/2
  o.bgf[2] = rqb;
  o.bgf[3] = bhb;
  o.bgf[4] = ibb;
  o.bgf[5] = pbf;
  o.bgf[6] = ppf;
  o.up[0] = 0.5f * v0;
  o.up[1] = 0.5f * v1;
  o.up[2] = 0.5f * v2;
  return o;
}

// Mixed-precision stage update of one node: r = -(1/J) (volume + lifts) in
// FP32, plus the background's right-hand side (stored in FP32) and the
// Coriolis source, all in FP32 (they join an FP32 increment); FP64 only in
// q += B dq.  Arrays are per node with stride NP between variables: rbg (3,
// background momentum rhs; 5, the full rhs of a moving background), qin (5),
// dqold (5) may be in shared or global memory; dq and qio are the node's
// global locations; qbg (5) the moving background's state (its Coriolis force
// is part of its rhs, so the source here acts on m - m_bg).  Returns true if
// the updated state is not finite or its density is not positive.
template <int NP, int BG>
__device__ __forceinline__ bool stage32(float (&r)[5], const float* rbg, const EsdgPhys& P,
                                        double y, const double* qin, const float* dqold, float* dq,
                                        double* qio, double rkA, double rkB, double dt,
                                        const double* qbg = nullptr) {
  if constexpr (BG == 2) {
#pragma unroll
    for (int v = 0; v < 5; v++) r[v] += rbg[v * NP];
  } else if constexpr (BG) {
    r[1] += rbg[0];
    r[2] += rbg[NP];
    r[3] += rbg[2 * NP];
  }
  if ((P.f0 != 0.0) || (P.beta != 0.0)) {
    const float f = esdg_d2f(P.f0 + P.beta * (y - P.y0));
    if constexpr (BG == 2) {
      r[1] = fmaf(f, esdg_d2f(qin[2 * NP] - qbg[2 * NP]), r[1]);
      r[2] = fmaf(-f, esdg_d2f(qin[NP] - qbg[NP]), r[2]);
    } else {
      r[1] = fmaf(f, esdg_d2f(qin[2 * NP]), r[1]);
      r[2] = fmaf(-f, esdg_d2f(qin[NP]), r[2]);
    }
  }
  const float A = esdg_d2f(rkA), B = esdg_d2f(rkB), dtf = esdg_d2f(dt);
  bool bad = false;
#pragma unroll
  for (int v = 0; v < 5; v++) {
    // the first stage (A = 0) does not read the register: a register left
    // non-finite by an earlier diverged run must not poison a new one
    const float dv = A == 0.0f ? dtf * r[v] : fmaf(A, dqold[(size_t)v * NP], dtf * r[v]);
    dq[(size_t)v * NP] = dv;
    const double qn = qin[(size_t)v * NP] + esdg_f2d(B * dv);
    qio[(size_t)v * NP] = qn;
    bad |= esdg_bad_state(qn, v == 0);
  }
  return bad;
}

}  // namespace esdg_vol
