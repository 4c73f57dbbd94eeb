// geometry.cu -- device construction of the mesh geometry and initial states.
//
// Node positions: uniform box elements, then the smooth warp of the mesh
// description; metric terms in Kopriva's conservative curl form
//   Ja^d_c = -e_d . curl_xi( X_l grad_xi X_m ),  (c, m, l) cyclic,
// with every reference derivative taken by the LGL differentiation matrix, and
// J = X_xi . (X_eta x X_zeta) (Section 3, the geometric factors G and G^s of
// Eq. (nm:semi)).  One CTA per element, one thread per node.
#include "dd.cuh"
#include "esdg_internal.cuh"

namespace {

// All geometry arithmetic runs in double-double and is rounded once: the curl
// form differentiates positions twice, so FP64 position round-off (relative to
// the element size) would reach the metric amplified by ~N^4.  Rounded from
// double-double, the metric terms are those of the exact node positions and
// agree on both sides of every face.
__global__ void k_geometry(EsdgGrid g, EsdgLGL L, EsdgPhys P, double* __restrict__ xo,
                           double* __restrict__ Jo, double* __restrict__ Jao,
                           double* __restrict__ vgeo, float* __restrict__ vgeo32) {
  extern __shared__ dd sg[];
  const int Nq = g.Nq, np = g.np;
  const int e = blockIdx.x;
  dd* X = sg;            // [3][np]
  dd* dX = X + 3 * np;   // [3 comp][3 dir][np]
  dd* V = dX + 9 * np;   // [3][np]
  dd* R1 = V + 3 * np;   // [3][Nq] 1-D node offsets from lo along each direction
  dd* S1 = R1 + 3 * Nq;  // [3][Nq] their warp sines sin(2 pi r / L)
  const int ex = e % g.K[0], ey = (e / g.K[0]) % g.K[1], ez = e / (g.K[0] * g.K[1]);
  const int eidx[3] = {ex, ey, ez};
  // the unwarped coordinates and the warp sines are functions of one 1-D index
  for (int it = threadIdx.x; it < 3 * Nq; it += blockDim.x) {
    const int d = it / Nq, i = it - d * Nq;
    const double Ld = g.hi[d] - g.lo[d];
    // offset from lo: L (e + (1 + xi)/2) / K of the whole box
    const dd xi = dd{L.xi[i], L.xi_lo[i]};
    dd t = dd_add(dd_make(1.0), xi);
    t = dd{0.5 * t.hi, 0.5 * t.lo};
    // the parent mesh's element index (a partition's elements are offset by eoff)
    t = dd_add(dd_make((double)(eidx[d] + g.eoff[d])), t);
    R1[it] = dd_div_d(dd_mul_d(t, Ld), (double)g.Kg[d]);
    if (g.warp != 0.0) S1[it] = dd_sinpi(dd_div_d(dd_mul_d(R1[it], 2.0), Ld));
  }
  __syncthreads();
  for (int n = threadIdx.x; n < np; n += blockDim.x) {
    const int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
    dd o[3] = {R1[ijk[0]], R1[Nq + ijk[1]], R1[2 * Nq + ijk[2]]};
    if (g.warp != 0.0) {
      const dd sv[3] = {S1[ijk[0]], S1[Nq + ijk[1]], S1[2 * Nq + ijk[2]]};
      const double Ld[3] = {g.hi[0] - g.lo[0], g.hi[1] - g.lo[1], g.hi[2] - g.lo[2]};
      o[0] = dd_add(o[0], dd_mul(dd_mul_d(sv[1], g.warp * Ld[0]), sv[2]));
      o[1] = dd_add(o[1], dd_mul(dd_mul_d(sv[2], g.warp * Ld[1]), sv[0]));
      o[2] = dd_add(o[2], dd_mul(dd_mul_d(sv[0], g.warp * Ld[2]), sv[1]));
    }
    for (int c = 0; c < 3; c++) {
      const dd Xc = dd_add(dd_make(g.lo[c]), o[c]);
      X[c * np + n] = Xc;
      xo[((size_t)e * 3 + c) * np + n] = Xc.hi;
    }
  }
  __syncthreads();
  // dX[c][d] = D_d X_c
  for (int n = threadIdx.x; n < np; n += blockDim.x) {
    const int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
    const int strides[3] = {1, Nq, Nq * Nq};
    for (int d = 0; d < 3; d++) {
      const int base = n - ijk[d] * strides[d];
      for (int c = 0; c < 3; c++) {
        dd s = dd_make(0.0);
        for (int m = 0; m < Nq; m++)
          s = dd_add(s, dd_mul(dd{L.D[ijk[d]][m], L.D_lo[ijk[d]][m]}, X[c * np + base + m * strides[d]]));
        dX[(c * 3 + d) * np + n] = s;
      }
    }
  }
  __syncthreads();
  // J = X_xi . (X_eta x X_zeta)
  for (int n = threadIdx.x; n < np; n += blockDim.x) {
    const dd a0 = dX[0 * np + n], a1 = dX[3 * np + n], a2 = dX[6 * np + n];  // d/dxi
    const dd b0 = dX[1 * np + n], b1 = dX[4 * np + n], b2 = dX[7 * np + n];  // d/deta
    const dd c0 = dX[2 * np + n], c1 = dX[5 * np + n], c2 = dX[8 * np + n];  // d/dzeta
    dd Jd = dd_mul(a0, dd_sub(dd_mul(b1, c2), dd_mul(b2, c1)));
    Jd = dd_add(Jd, dd_mul(a1, dd_sub(dd_mul(b2, c0), dd_mul(b0, c2))));
    Jd = dd_add(Jd, dd_mul(a2, dd_sub(dd_mul(b0, c1), dd_mul(b1, c0))));
    const double J = Jd.hi;
    const double z = X[2 * np + n].hi, z0 = X[2 * np].hi;
    Jo[(size_t)e * np + n] = J;
    vgeo[((size_t)e * ESDG_NVGEO + 9) * np + n] = 1.0 / J;
    vgeo[((size_t)e * ESDG_NVGEO + 10) * np + n] = P.g * z;
    vgeo32[((size_t)e * ESDG_NVGEO + 9) * np + n] = (float)(1.0 / J);
    // FP32 geometry carries (phi - phi_0)/2, phi_0 at the element's first node
    // (the mixed kernels' pair geopotential)
    vgeo32[((size_t)e * ESDG_NVGEO + 10) * np + n] = 0.5f * (float)(P.g * z - P.g * z0);
  }
  // curl form, one physical component c at a time
  for (int c = 0; c < 3; c++) {
    const int m = (c + 1) % 3, l = (c + 2) % 3;
    __syncthreads();
    // X_l relative to the element's first node: the curl of (const * grad X_m)
    // vanishes identically
    const dd xl0 = X[l * np];
    for (int n = threadIdx.x; n < np; n += blockDim.x)
      for (int d = 0; d < 3; d++) V[d * np + n] = dd_mul(dd_sub(X[l * np + n], xl0), dX[(m * 3 + d) * np + n]);
    __syncthreads();
    for (int n = threadIdx.x; n < np; n += blockDim.x) {
      const int ijk[3] = {n % Nq, (n / Nq) % Nq, n / (Nq * Nq)};
      const int strides[3] = {1, Nq, Nq * Nq};
      for (int d = 0; d < 3; d++) {
        // (curl V)_d = d_p V_q - d_q V_p with (d, p, q) cyclic
        const int p = (d + 1) % 3, q = (d + 2) % 3;
        const int bp = n - ijk[p] * strides[p], bq = n - ijk[q] * strides[q];
        dd s1 = dd_make(0.0), s2 = dd_make(0.0);
        for (int k = 0; k < Nq; k++) {
          s1 = dd_add(s1, dd_mul(dd{L.D[ijk[p]][k], L.D_lo[ijk[p]][k]}, V[q * np + bp + k * strides[p]]));
          s2 = dd_add(s2, dd_mul(dd{L.D[ijk[q]][k], L.D_lo[ijk[q]][k]}, V[p * np + bq + k * strides[q]]));
        }
        const double ja = -dd_sub(s1, s2).hi;
        Jao[(((size_t)e * 3 + d) * 3 + c) * np + n] = ja;
        vgeo[((size_t)e * ESDG_NVGEO + d * 3 + c) * np + n] = 0.5 * ja;
        vgeo32[((size_t)e * ESDG_NVGEO + d * 3 + c) * np + n] = (float)(0.5 * ja);
      }
    }
  }
}

// Face normals from the metric of the element on the face's "-" side (or the
// "+" side at a low wall): nhat = Ja^d / |Ja^d| points along +d; s / w_end is
// the lift scaling; phi the geopotential at the face node.
__global__ void k_face_geometry(EsdgGrid g, EsdgLGL L, EsdgPhys P, const double* __restrict__ x,
                                const double* __restrict__ Ja, double* __restrict__ fgeo) {
  const int Nq = g.Nq, nf2 = Nq * Nq;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= g.nfaces * nf2) return;
  const long long f = tid / nf2;
  const int fn = (int)(tid - f * nf2);
  int d = 0;
  while (d < 2 && f >= g.face_off[d + 1]) d++;
  int o1, o2;
  esdg_others(d, o1, o2);
  long long r = f - g.face_off[d];
  const int a = (int)(r % g.K[o1]);
  r /= g.K[o1];
  const int b = (int)(r % g.K[o2]);
  const int Pl = (int)(r / g.K[o2]);
  int idx[3];
  idx[o1] = a;
  idx[o2] = b;
  int side_end;
  if (Pl > 0 || g.periodic[d]) {
    idx[d] = (Pl - 1 + g.K[d]) % g.K[d];
    side_end = g.N;
  } else {
    idx[d] = 0;
    side_end = 0;
  }
  const int e = idx[0] + g.K[0] * (idx[1] + g.K[1] * idx[2]);
  int ijk[3];
  ijk[d] = side_end;
  ijk[o1] = fn % Nq;
  ijk[o2] = fn / Nq;
  const int n = esdg_node(Nq, ijk[0], ijk[1], ijk[2]);
  const double j0 = Ja[(((size_t)e * 3 + d) * 3 + 0) * g.np + n];
  const double j1 = Ja[(((size_t)e * 3 + d) * 3 + 1) * g.np + n];
  const double j2 = Ja[(((size_t)e * 3 + d) * 3 + 2) * g.np + n];
  const double s = sqrt(j0 * j0 + j1 * j1 + j2 * j2);
  double* o = fgeo + (size_t)f * 5 * nf2;
  o[0 * nf2 + fn] = j0 / s;
  o[1 * nf2 + fn] = j1 / s;
  o[2 * nf2 + fn] = j2 / s;
  o[3 * nf2 + fn] = s / L.w[g.N];
  o[4 * nf2 + fn] = P.g * x[((size_t)e * 3 + 2) * g.np + n];
}

// Section 5.1 over an isentropic hydrostatic background: the cosine bubble of
// Eq. (smooth-rb-ic) (sharp = 0) or the step of Eq. (sharp-rb-ic) (sharp = 1) in theta;
// Exner = 1 - g z/(cp theta0), p = p0 Exner^(cp/R), T = theta Exner, rho = p/(R T).
__global__ void k_bubble(EsdgGrid g, EsdgPhys P, const double* __restrict__ x, double theta0,
                         double amp, double cx, double cy, double cz, double radius, int sharp,
                         double* __restrict__ q) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double X = x[(e * 3 + 0) * np + n], Y = x[(e * 3 + 1) * np + n], Z = x[(e * 3 + 2) * np + n];
  const double cp = P.gamma * P.R / (P.gamma - 1.0);
  const double r = sqrt((X - cx) * (X - cx) + (Y - cy) * (Y - cy) + (Z - cz) * (Z - cz));
  const double dth = (r <= radius) ? (sharp ? amp : amp * 0.5 * (1.0 + cospi(r / radius))) : 0.0;
  const double ex = 1.0 - P.g * Z / (cp * theta0);
  const double p = P.p0 * pow(ex, cp / P.R);
  const double rho = p / (P.R * (theta0 + dth) * ex);
  double* qe = q + e * 5 * np;
  qe[0 * np + n] = rho;
  qe[1 * np + n] = 0.0;
  qe[2 * np + n] = 0.0;
  qe[3 * np + n] = 0.0;
  qe[4 * np + n] = p / (P.gamma - 1.0) + rho * P.g * Z;
}

// Synthetic channel: ln p = ln p0 - z/H(y), H = H0 + dH (1 - tanh((y - yc)/delta))/2,
// rho = p/(g H), geostrophic u = -g z H'(y)/(f H), plus a Gaussian of amplitude up in u
// (1 m/s in the channel workload; 0 gives the balanced jet alone).
__global__ void k_channel(EsdgGrid g, EsdgPhys P, const double* __restrict__ x,
                          double* __restrict__ q, double up) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double H0 = 7500.0, dH = 120.0, delta = 600e3, yc = 3000e3;
  const double xp = 2000e3, yp = 2500e3, Lp = 600e3;
  const double X = x[(e * 3 + 0) * np + n], Y = x[(e * 3 + 1) * np + n], Z = x[(e * 3 + 2) * np + n];
  const double th = tanh((Y - yc) / delta);
  const double H = H0 + dH * 0.5 * (1.0 - th);
  const double dHdy = -dH * (1.0 - th * th) / (2.0 * delta);
  const double f = P.f0 + P.beta * (Y - P.y0);
  const double p = P.p0 * exp(-Z / H);
  const double rho = p / (P.g * H);
  double u = -P.g * Z * dHdy / (f * H);
  u += up * exp(-((X - xp) * (X - xp) + (Y - yp) * (Y - yp)) / (Lp * Lp));
  double* qe = q + e * 5 * np;
  qe[0 * np + n] = rho;
  qe[1 * np + n] = rho * u;
  qe[2 * np + n] = 0.0;
  qe[3 * np + n] = 0.0;
  qe[4 * np + n] = p / (P.gamma - 1.0) + 0.5 * rho * u * u + rho * P.g * Z;
}

// Background of the mixed-precision path: rho_bg, b_bg = rho/(2p) and p_bg of a
// given state, and the same state at rest, (rho, 0, 0, 0, p/(gamma-1) + rho phi).
__global__ void k_background(EsdgGrid g, EsdgPhys P, const double* __restrict__ vgeo,
                             const double* __restrict__ q, double* __restrict__ bg,
                             double* __restrict__ q0) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double* qe = q + e * 5 * np;
  const double phi = vgeo[(e * ESDG_NVGEO + 10) * np + n];
  const double rho = qe[n];
  const double ke = 0.5 * (qe[np + n] * qe[np + n] + qe[2 * np + n] * qe[2 * np + n] +
                           qe[3 * np + n] * qe[3 * np + n]) / rho;
  const double p = (P.gamma - 1.0) * (qe[4 * np + n] - ke - rho * phi);
  bg[(e * 3 + 0) * np + n] = rho;
  bg[(e * 3 + 1) * np + n] = rho / (2.0 * p);
  bg[(e * 3 + 2) * np + n] = p;
  double* o = q0 + e * 5 * np;
  o[n] = rho;
  o[np + n] = 0.0;
  o[2 * np + n] = 0.0;
  o[3 * np + n] = 0.0;
  o[4 * np + n] = fma(rho, phi, p / (P.gamma - 1.0));
}

__global__ void k_background_state(EsdgGrid g, EsdgPhys P, const double* __restrict__ vgeo,
                                   const double* __restrict__ bg, double* __restrict__ q0) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double phi = vgeo[(e * ESDG_NVGEO + 10) * np + n];
  const double rho = bg[(e * 3 + 0) * np + n], p = bg[(e * 3 + 2) * np + n];
  double* o = q0 + e * 5 * np;
  o[n] = rho;
  o[np + n] = 0.0;
  o[2 * np + n] = 0.0;
  o[3 * np + n] = 0.0;
  o[4 * np + n] = fma(rho, phi, p / (P.gamma - 1.0));
}

// The mixed volume kernels' copy of the background: bg3 = (rho_bg, E_bg, phi)
// in FP64, E_bg = p_bg/(gamma - 1) + rho_bg phi the background's total energy
// at rest (the expression of k_background), for the exact FP64 differences
// rho - rho_bg and E - E_bg, with the geopotential beside them so that one
// bulk copy brings all three; bgp = (rho_bg/4, b_bg/2, 1/b_bg, p_bg) in FP32, the
// background's node fields of the FP32 pair loop, converted once here instead
// of at every stage.
__global__ void k_background_vol(EsdgGrid g, EsdgPhys P, const double* __restrict__ vgeo,
                                 const double* __restrict__ bg, double* __restrict__ bg3,
                                 float* __restrict__ bgp) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double phi = vgeo[(e * ESDG_NVGEO + 10) * np + n];
  const double rho = bg[(e * 3 + 0) * np + n], b = bg[(e * 3 + 1) * np + n],
               p = bg[(e * 3 + 2) * np + n];
  bg3[(e * 3 + 0) * np + n] = rho;
  bg3[(e * 3 + 1) * np + n] = fma(rho, phi, p / (P.gamma - 1.0));
  bg3[(e * 3 + 2) * np + n] = phi;
  bgp[(e * 4 + 0) * np + n] = __double2float_rn(0.25 * rho);
  bgp[(e * 4 + 1) * np + n] = __double2float_rn(0.5 * b);
  bgp[(e * 4 + 2) * np + n] = __double2float_rn(1.0 / b);
  bgp[(e * 4 + 3) * np + n] = __double2float_rn(p);
}

// u_bg = m_bg / rho_bg of a moving background, rounded to FP32
__global__ void k_background_velocity(EsdgGrid g, const double* __restrict__ bgq,
                                      float* __restrict__ bgu) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int np = g.np;
  if (tid >= (long long)g.E * np) return;
  const long long e = tid / np;
  const int n = (int)(tid - e * np);
  const double* qe = bgq + e * 5 * np;
  const double ir = 1.0 / qe[n];
  for (int d = 0; d < 3; d++) bgu[(e * 3 + d) * np + n] = __double2float_rn(qe[(1 + d) * np + n] * ir);
}

__global__ void k_to_f32(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __double2float_rn(src[i]);
}

}  // namespace

cudaError_t esdg_launch_background_vol(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                       const double* bg, double* bg3, float* bgp, cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  if (nt == 0) return cudaSuccess;
  k_background_vol<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, P, vgeo, bg, bg3, bgp);
  return cudaGetLastError();
}

cudaError_t esdg_launch_background_velocity(const EsdgGrid& g, const double* bgq, float* bgu,
                                            cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  if (nt == 0) return cudaSuccess;
  k_background_velocity<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, bgq, bgu);
  return cudaGetLastError();
}

cudaError_t esdg_launch_to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t esdg_launch_background_state(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                         const double* bg, double* q0, cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  k_background_state<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, P, vgeo, bg, q0);
  return cudaGetLastError();
}

cudaError_t esdg_launch_background(const EsdgGrid& g, const EsdgPhys& P, const double* vgeo,
                                   const double* q, double* bg, double* q0, cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  k_background<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, P, vgeo, q, bg, q0);
  return cudaGetLastError();
}

cudaError_t esdg_launch_geometry(const EsdgGrid& g, const EsdgLGL& L, double* x, double* J,
                                 double* Ja, double* vgeo, float* vgeo32, double* fgeo,
                                 const EsdgPhys& P, cudaStream_t s) {
  const size_t smem = sizeof(dd) * (15 * (size_t)g.np + 6 * (size_t)g.Nq);
  if (smem > 48 * 1024) {
    cudaError_t err = cudaFuncSetAttribute(k_geometry, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
  }
  const int thr = g.np < 256 ? ((g.np + 31) / 32) * 32 : 256;
  k_geometry<<<g.E, thr, smem, s>>>(g, L, P, x, J, Ja, vgeo, vgeo32);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const long long nt = g.nfaces * g.Nq * g.Nq;
  if (nt > 0) {
    k_face_geometry<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, L, P, x, Ja, fgeo);
    err = cudaGetLastError();
  }
  return err;
}

cudaError_t esdg_launch_bubble(const EsdgGrid& g, const EsdgPhys& P, const double* x, double theta0,
                               double amp, const double* c, double radius, int sharp, double* q,
                               cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  k_bubble<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, P, x, theta0, amp, c[0], c[1], c[2],
                                                         radius, sharp, q);
  return cudaGetLastError();
}

cudaError_t esdg_launch_channel(const EsdgGrid& g, const EsdgPhys& P, const double* x, double* q,
                                double amp, cudaStream_t s) {
  const long long nt = (long long)g.E * g.np;
  k_channel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(g, P, x, q, amp);
  return cudaGetLastError();
}
