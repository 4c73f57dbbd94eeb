// checks.cu -- test hook that runs the hand-written numeric helpers of the
// kernels (esdg_internal.cuh) on caller-owned device arrays, so that tests can
// hold them to the IEEE-754 operations they stand in for.
#include "../../include/es_dg.h"
#include "esdg_internal.cuh"

namespace {

__global__ void k_numeric(int which, const void* __restrict__ in, void* __restrict__ out,
                          long long n, int k) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double* xd = static_cast<const double*>(in);
    const float* xf = static_cast<const float*>(in);
    double* yd = static_cast<double*>(out);
    float* yf = static_cast<float*>(out);
    switch (which) {
      case ES_DG_NUM_D2F: yf[i] = esdg_d2f(xd[i]); break;
      case ES_DG_NUM_F2D: yd[i] = esdg_f2d(xf[i]); break;
      case ES_DG_NUM_LDEXP: yd[i] = esdg_ldexp(xd[i], k); break;
      case ES_DG_NUM_RCP: yd[i] = esdg_rcp(xd[i]); break;
      case ES_DG_NUM_RCP_LO: yd[i] = esdg_rcp_lo(xd[i]); break;
      case ES_DG_NUM_D2F_TAIL: yf[i] = esdg_d2f_tail(xd[i]); break;
      case ES_DG_NUM_F2D_POS: yd[i] = esdg_f2d_pos(xf[i]); break;
      default: break;
    }
  }
}

}  // namespace

extern "C" int es_dg_debug_numeric(int which, const void* in, void* out, long long n, int k,
                                   void* cuda_stream) {
  if (which < ES_DG_NUM_D2F || which > ES_DG_NUM_F2D_POS || n < 0 || (n > 0 && (!in || !out)))
    return ES_DG_EINVAL;
  if (n == 0) return ES_DG_OK;
  const long long blocks = (n + 255) / 256;
  k_numeric<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)cuda_stream>>>(
      which, in, out, n, k);
  return cudaGetLastError() == cudaSuccess ? ES_DG_OK : ES_DG_ECUDA;
}
