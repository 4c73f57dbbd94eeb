// reduce.cu -- global reductions over the state: the CFL time step and the
// conservation/entropy integrals (the monitors of Section 5.2).
//
// Two passes with a scratch buffer: pass 1 writes one partial per element
// (fixed order inside the CTA), pass 2 folds the partials in one CTA in a fixed
// order, so results are reproducible run to run.
#include "esdg_internal.cuh"

namespace {

constexpr int RT = 256;  // threads of the second pass

__device__ __forceinline__ double block_reduce(double v, double* sh, bool take_min) {
  // warp level, then across warps through shared memory
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_down_sync(0xffffffffu, v, o);
    v = take_min ? fmin(v, w) : v + w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (threadIdx.x == 0) {
    double r = sh[0];
    for (int k = 1; k < nw; k++) r = take_min ? fmin(r, sh[k]) : r + sh[k];
    sh[0] = r;
  }
  __syncthreads();
  return sh[0];
}

// one CTA per element: the largest reference-space signal speed
//   lambda = max_n max_d (|u . Ja^d| + c |Ja^d|) / J;
// the time step is C (xi_1 - xi_0) / max_e lambda_e (on an affine element this
// is the node-spacing rule C h (xi_1 - xi_0) / (2 (|u_d| + c))).  The partial
// stored is 1/lambda so that the fold takes a minimum.
__global__ void k_cfl_elem(EsdgGrid g, EsdgLGL L, EsdgPhys P, const double* __restrict__ q,
                           const double* __restrict__ x, const double* __restrict__ J,
                           const double* __restrict__ Ja, double* __restrict__ part) {
  __shared__ double sh[32];
  const int e = blockIdx.x, np = g.np;
  double lmax = 0.0;
  for (int n = threadIdx.x; n < np; n += blockDim.x) {
    const double* qe = q + (size_t)e * 5 * np;
    const double rho = qe[n], ir = 1.0 / rho;
    const double u0 = qe[np + n] * ir, u1 = qe[2 * np + n] * ir, u2 = qe[3 * np + n] * ir;
    const double z = x[((size_t)e * 3 + 2) * np + n];
    const double p = (P.gamma - 1.0) *
                     (qe[4 * np + n] - 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2) - rho * P.g * z);
    const double cs = sqrt(P.gamma * p * ir);
    const double iJ = 1.0 / J[(size_t)e * np + n];
    for (int d = 0; d < 3; d++) {
      const double* ja = Ja + (((size_t)e * 3 + d) * 3) * np + n;
      const double a0 = ja[0], a1 = ja[np], a2 = ja[2 * np];
      const double lam = (fabs(u0 * a0 + u1 * a1 + u2 * a2) + cs * sqrt(a0 * a0 + a1 * a1 + a2 * a2)) * iJ;
      lmax = fmax(lmax, lam);
    }
  }
  lmax = -block_reduce(-lmax, sh, true);
  if (threadIdx.x == 0) part[e] = 1.0 / lmax;
}

// one CTA per element: quadrature of rho, E and eta = -rho s/(gamma-1)
__global__ void k_integrals_elem(EsdgGrid g, EsdgLGL L, EsdgPhys P, const double* __restrict__ q,
                                 const double* __restrict__ J, const double* __restrict__ x,
                                 double* __restrict__ part) {
  __shared__ double sh[32];
  const int e = blockIdx.x, np = g.np, Nq = g.Nq;
  double m = 0.0, en = 0.0, ent = 0.0;
  for (int n = threadIdx.x; n < np; n += blockDim.x) {
    const double* qe = q + (size_t)e * 5 * np;
    const double wJ = L.w[n % Nq] * L.w[(n / Nq) % Nq] * L.w[n / (Nq * Nq)] * J[(size_t)e * np + n];
    const double rho = qe[n];
    const double ke = 0.5 * (qe[np + n] * qe[np + n] + qe[2 * np + n] * qe[2 * np + n] +
                             qe[3 * np + n] * qe[3 * np + n]) / rho;
    const double z = x[((size_t)e * 3 + 2) * np + n];
    const double p = (P.gamma - 1.0) * (qe[4 * np + n] - ke - rho * P.g * z);
    m += wJ * rho;
    en += wJ * qe[4 * np + n];
    ent += wJ * (-rho * (log(p) - P.gamma * log(rho)) / (P.gamma - 1.0));
  }
  m = block_reduce(m, sh, false);
  en = block_reduce(en, sh, false);
  ent = block_reduce(ent, sh, false);
  if (threadIdx.x == 0) {
    part[(size_t)e * 3 + 0] = m;
    part[(size_t)e * 3 + 1] = en;
    part[(size_t)e * 3 + 2] = ent;
  }
}

// fold `n` partials with stride `stride` (component c) into out[c]
__global__ void k_fold(const double* __restrict__ part, int n, int stride, int ncomp, int take_min,
                       double* __restrict__ out) {
  __shared__ double sh[32];
  for (int c = 0; c < ncomp; c++) {
    double v = take_min ? 1e300 : 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const double w = part[(size_t)k * stride + c];
      v = take_min ? fmin(v, w) : v + w;
    }
    v = block_reduce(v, sh, take_min != 0);
    if (threadIdx.x == 0) out[c] = v;
    __syncthreads();
  }
}

}  // namespace

size_t esdg_reduce_scratch(const EsdgGrid& g) { return (size_t)g.E * 3; }

cudaError_t esdg_launch_cfl(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, const double* q,
                            const double* x, const double* J, const double* Ja, double* scratch,
                            double* out, cudaStream_t s) {
  const int thr = g.np >= 256 ? 256 : ((g.np + 31) / 32) * 32;
  k_cfl_elem<<<g.E, thr, 0, s>>>(g, L, P, q, x, J, Ja, scratch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_fold<<<1, RT, 0, s>>>(scratch, g.E, 1, 1, 1, out);
  return cudaGetLastError();
}

cudaError_t esdg_launch_integrals(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                  const double* q, const double* J, const double* x,
                                  double* scratch, double* out, cudaStream_t s) {
  const int thr = g.np >= 256 ? 256 : ((g.np + 31) / 32) * 32;
  k_integrals_elem<<<g.E, thr, 0, s>>>(g, L, P, q, J, x, scratch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_fold<<<1, RT, 0, s>>>(scratch, g.E, 3, 3, 0, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the integrals reduction (es_dg_integrals_noalloc).
//
// Some callers cannot allocate device memory at all: code running under a
// memory pool it does not own, inside a framework that forbids cudaMalloc on
// its hot path, or in a process whose allocator is already exhausted.  For
// them the per-element partial sums live in the file-scope array below instead
// of a handle's scratch buffer.  The array is created with the module on every
// device that loads this library and stays there until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

#include "../../include/es_dg.h"

namespace {

static __device__ __align__(256) double g_noalloc_partials[3 * ES_DG_NOALLOC_MAX_ELEMS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of g_noalloc_partials on the current device.  In host code the
// symbol is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current.  It is looked up again on
// every call made while the stream is not capturing (a device reset reloads
// the module, possibly at another address); a call made during a capture uses
// the address found by the last call outside one.
int noalloc_scratch(cudaStream_t stream, double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return ES_DG_ECUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return ES_DG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone || !g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return ES_DG_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_addr[dev];
  return ES_DG_OK;
}

}  // namespace

extern "C" int es_dg_integrals_noalloc(const es_dg_mesh* mesh, int N, const es_dg_physics* physics,
                                       const double* q, const double* J, const double* x,
                                       double* out3, void* cuda_stream) {
  if (!mesh || !q || !J || !x || !out3 || N < 1 || N > 7) return ES_DG_EINVAL;
  if (mesh->kx < 1 || mesh->ky < 1 || mesh->kz < 1) return ES_DG_EINVAL;
  const long long E = (long long)mesh->kx * mesh->ky * mesh->kz;
  if (E > ES_DG_NOALLOC_MAX_ELEMS) return ES_DG_EINVAL;  // beyond the static scratch
  EsdgGrid g{};
  g.K[0] = mesh->kx;
  g.K[1] = mesh->ky;
  g.K[2] = mesh->kz;
  g.N = N;
  g.Nq = N + 1;
  g.np = g.Nq * g.Nq * g.Nq;
  g.E = (int)E;
  EsdgLGL L;
  if (esdg_lgl_build(N, &L)) return ES_DG_EINVAL;
  EsdgPhys P{1.4, 9.81, 287.0, 1.0e5, 0.0, 0.0, 0.0, 1, 0.0, 0.0};
  if (physics) {
    P.gamma = physics->gamma;
    P.g = physics->g;
    P.R = physics->R;
    P.p0 = physics->p0;
    P.f0 = physics->f0;
    P.beta = physics->beta;
    P.y0 = physics->y0;
    P.dissipation = physics->dissipation;
  }
  // the checks es_dg_create applies: a bad gas constant would make every
  // integral NaN without any error being reported
  if (!(P.gamma > 1.0) || !(P.R > 0.0) || !(P.p0 > 0.0)) return ES_DG_EINVAL;
  esdg_phys_derive(&P);
  double* scratch = nullptr;
  int st = noalloc_scratch((cudaStream_t)cuda_stream, &scratch);
  if (st) return st;
  // every partial the fold reads (the first E triples) is written by this
  // call, so nothing needs clearing between calls
  cudaError_t e = esdg_launch_integrals(g, L, P, q, J, x, scratch, out3, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ES_DG_ENOMEM : ES_DG_ECUDA;
  return ES_DG_OK;
}
