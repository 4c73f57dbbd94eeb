// api.cu -- the C ABI of include/es_dg.h: handle management, buffers and launch
// sequences.  All arithmetic happens in the kernels; this file only validates
// arguments, owns device memory and orders launches on the handle's stream.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/es_dg.h"
#include "esdg_internal.cuh"

namespace {

// Carpenter & Kennedy (1994), five-stage fourth-order 2N-storage coefficients
const double kRkA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                        -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRkB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                        1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                        2277821191437.0 / 14882151754819.0};

}  // namespace

struct es_dg {
  EsdgGrid g;
  EsdgLGL L;
  EsdgPhys P;
  int mixed;
  cudaStream_t stream;
  es_dg_allocator alloc;
  int has_alloc;
  std::vector<void*> blocks;
  size_t bytes;
  double* q;
  void* dq;
  double *x, *J, *Ja, *vgeo, *fgeo;
  float* vgeo32;
  void* fflux;
  double* rhs;      // lazily allocated
  double* qtmp;     // lazily allocated
  double* scratch;  // reductions
  double* result;   // small device result slots (3 doubles, then the status word)
  int* status;      // set by a stage update whose new state is not finite or has a
                    // non-positive density; read and cleared by es_dg_sync
  // mixed precision relative to a hydrostatic background
  int has_bg;
  double* bg;       // [E][3][np] rho_bg, b_bg, p_bg
  double* rhs_bg;   // [E][3][np] FP64 momentum right-hand side of the background at rest
  double* fflux64;  // FP64 face fluxes for evaluating that right-hand side
  // the mixed volume kernels' copy: bg3 [E][3][np] rho_bg, E_bg, phi; bgp [E][4][np] FP32
  // rho_bg/4, b_bg/2, 1/b_bg, p_bg; rhs_bg32 [E][3][np] the momentum rhs in FP32
  double* bg3;
  float* bgp;
  float* rhs_bg32;
  // a moving background (carries a flow; whole meshes only): its state bgq
  // [E][5][np], u_bg in FP32 bgu [E][3][np], its full right-hand side in FP32
  // rhs_bgm32 [E][5][np]
  int bg_moving;
  double* bgq;
  float* bgu;
  float* rhs_bgm32;
  // a partition's trace buffers (caller-owned device memory; [0] low x plane, [1] high)
  double* tr_send[2];
  double* tr_recv[2];
  // a mixed partition evaluates its background's right-hand side at its first stage,
  // once its neighbours' background values have arrived with the traces
  int bg_pending;
  // es_dg_partitions_step: this partition's own stream and the events ordering it
  // against its neighbours (created on first use)
  cudaStream_t pstream;
  cudaEvent_t ev_packed, ev_sent, ev_faced, ev_join;
  // configuration generation (unique across handles): renewed whenever what a
  // captured step launches could change (traces, background)
  long long gen;
  // the captured LSRK step of the partitions this handle leads (parts[0]), its
  // time step and the partitions and generations it was captured for
  cudaGraphExec_t pexec;
  double pexec_dt;
  std::vector<es_dg_t*> pexec_parts;
  std::vector<long long> pexec_gens;
};

namespace {

long long next_gen() {
  static std::atomic<long long> counter{0};
  return ++counter;
}

void touch(es_dg_t* h) { h->gen = next_gen(); }

int dev_alloc(es_dg_t* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  if (h->has_alloc) {
    *p = h->alloc.alloc(bytes, h->alloc.ctx);
    if (!*p) return ES_DG_ENOMEM;
  } else {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return ES_DG_ENOMEM;
    }
  }
  h->blocks.push_back(*p);
  h->bytes += bytes;
  return ES_DG_OK;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ES_DG_OK;
  if (e == cudaErrorMemoryAllocation) return ES_DG_ENOMEM;
  return ES_DG_ECUDA;
}

// The grid of a whole mesh (x_end < 0) or of its partition of x element
// layers [x_begin, x_end): the partition keeps the parent's box and element
// counts for its node positions; a cut x plane becomes remote, and a periodic
// x wraps through the traces (unless one partition holds the whole mesh).
int build_grid(const es_dg_mesh* m, int N, EsdgGrid* g, int x_begin = 0, int x_end = -1) {
  if (!m || N < 1 || N > 7) return ES_DG_EINVAL;
  int K[3] = {m->kx, m->ky, m->kz};
  int per[3] = {m->periodic[0] ? 1 : 0, m->periodic[1] ? 1 : 0, m->periodic[2] ? 1 : 0};
  for (int d = 0; d < 3; d++)
    if (K[d] < 1 || !(m->hi[d] > m->lo[d])) return ES_DG_EINVAL;
  std::memset(g, 0, sizeof(*g));
  for (int d = 0; d < 3; d++) g->Kg[d] = K[d];
  if (x_end >= 0) {
    if (x_begin < 0 || x_end > K[0] || x_begin >= x_end) return ES_DG_EINVAL;
    if (x_begin > 0 || x_end < K[0]) {
      g->remote[0] = (x_begin > 0 || per[0]) ? 1 : 0;
      g->remote[1] = (x_end < K[0] || per[0]) ? 1 : 0;
      per[0] = 0;
      g->eoff[0] = x_begin;
      K[0] = x_end - x_begin;
    }
  }
  long long E = 1;
  for (int d = 0; d < 3; d++) E *= K[d];
  if (E > (1LL << 30) || !(m->warp >= 0.0 && m->warp < 0.15)) return ES_DG_EINVAL;
  for (int d = 0; d < 3; d++) {
    g->K[d] = K[d];
    g->periodic[d] = per[d];
    g->lo[d] = m->lo[d];
    g->hi[d] = m->hi[d];
    g->nplanes[d] = g->periodic[d] ? K[d] : K[d] + 1;
  }
  g->warp = m->warp;
  g->N = N;
  g->Nq = N + 1;
  g->np = g->Nq * g->Nq * g->Nq;
  g->E = (int)E;
  long long off = 0;
  for (int d = 0; d < 3; d++) {
    int o1, o2;
    esdg_others(d, o1, o2);
    g->face_off[d] = off;
    off += (long long)g->nplanes[d] * K[o1] * K[o2];
  }
  g->nfaces = off;
  return ES_DG_OK;
}

int ensure_rhs_buffers(es_dg_t* h) {
  const size_t n = (size_t)h->g.E * 5 * h->g.np;
  int st = ES_DG_OK;
  if (!h->rhs) st = dev_alloc(h, (void**)&h->rhs, n * sizeof(double));
  if (st == ES_DG_OK && !h->qtmp) st = dev_alloc(h, (void**)&h->qtmp, n * sizeof(double));
  return st;
}

EsdgVolArgs vol_args(es_dg_t* h, const double* q_in, double* rhs_out) {
  EsdgVolArgs a;
  a.q_in = q_in;
  a.q_io = h->q;
  a.dq = h->dq;
  a.rhs = rhs_out;
  a.vgeo = h->mixed ? (const void*)h->vgeo32 : (const void*)h->vgeo;
  a.vgeo64 = h->vgeo;
  a.fflux = h->fflux;
  a.x = h->x;
  a.bg = (h->mixed && h->has_bg) ? h->bg3 : nullptr;
  a.bgp = h->bgp;
  a.rhs_bg = h->rhs_bg32;
  const bool moving = h->mixed && h->has_bg && h->bg_moving;
  a.bgq = moving ? h->bgq : nullptr;
  a.bgu = moving ? h->bgu : nullptr;
  a.rhs_bgm = moving ? h->rhs_bgm32 : nullptr;
  a.rkA = 0.0;
  a.rkB = 0.0;
  a.dt = 0.0;
  a.status = h->status;
  return a;
}

bool is_partition(const es_dg_t* h) { return h->g.remote[0] || h->g.remote[1]; }

// every remote plane of a partition has its received trace
bool traces_ready(const es_dg_t* h) {
  for (int s = 0; s < 2; s++)
    if (h->g.remote[s] && !h->tr_recv[s]) return false;
  return true;
}

// doubles per face node in a trace: the state, and for mixed handles rho_bg and p_bg
int trace_nv(const es_dg_t* h) { return h->mixed ? 7 : 5; }

size_t trace_doubles(const es_dg_t* h) {
  return (size_t)h->g.K[1] * h->g.K[2] * trace_nv(h) * h->g.Nq * h->g.Nq;
}

EsdgTraces traces_of(const es_dg_t* h) {
  return EsdgTraces{h->tr_recv[0], h->tr_recv[1], trace_nv(h), 0};
}

int resolve_background(es_dg_t* h);

// The interface fluxes of one class of faces for state q_in: 0 every face, 1 the
// faces whose outside state needs no trace, 2 the faces of the remote planes.
// x faces come first, plane by plane (plane 0 is a partition's low cut, the last
// x plane its high cut), then the y and z faces.
enum { FACES_ALL = 0, FACES_INTERIOR = 1, FACES_CUT = 2 };
int launch_faces(es_dg_t* h, const double* q_in, int which) {
  const bool moving = h->mixed && h->has_bg && h->bg_moving;
  const double* bg = (h->mixed && h->has_bg) ? h->bg : nullptr;
  const EsdgTraces tr = traces_of(h);
  auto run = [&](long long f0, long long f1) {
    return esdg_launch_face(h->g, h->P, h->mixed, q_in, h->fgeo, h->fflux, h->stream, bg, tr,
                            moving ? h->bgq : nullptr, f0, f1);
  };
  const long long plane = (long long)h->g.K[1] * h->g.K[2];
  const long long x0 = h->g.face_off[0], x1 = h->g.face_off[1];
  const long long lo = h->g.remote[0] ? plane : 0, hi = h->g.remote[1] ? plane : 0;
  cudaError_t e = cudaSuccess;
  if (which == FACES_ALL) {
    e = run(0, -1);
  } else if (which == FACES_INTERIOR) {
    e = run(x0 + lo, x1 - hi);
    if (e == cudaSuccess) e = run(x1, -1);
  } else {
    if (lo) e = run(x0, x0 + lo);
    if (e == cudaSuccess && hi) e = run(x1 - hi, x1);
  }
  return cuda_status(e);
}

// face fluxes then volume (+ lift, source, optional RK update) for state q_in
int launch_stage(es_dg_t* h, const double* q_in, int mode, double* rhs_out, double A, double B,
                 double dt) {
  if (!traces_ready(h)) return ES_DG_EINVAL;
  if (h->bg_pending) {
    const int st = resolve_background(h);
    if (st) return st;
  }
  const int stf = launch_faces(h, q_in, FACES_ALL);
  if (stf) return stf;
  EsdgVolArgs a = vol_args(h, q_in, rhs_out);
  a.rkA = A;
  a.rkB = B;
  a.dt = dt;
  const cudaError_t e = esdg_launch_volume(h->g, h->L, h->P, h->mixed, mode, a, h->stream);
  return cuda_status(e);
}

// Set the mixed path's hydrostatic background from state q_dev (device): store
// rho_bg and b_bg, and evaluate the right-hand side of the background at rest
// once with the FP64 kernels.
int set_background_dev(es_dg_t* h, const double* q_dev) {
  const size_t E = h->g.E, np = h->g.np, nf2 = (size_t)h->g.Nq * h->g.Nq;
  int st = ensure_rhs_buffers(h);
  if (!st && !h->bg) st = dev_alloc(h, (void**)&h->bg, E * 3 * np * sizeof(double));
  if (!st && !h->rhs_bg) st = dev_alloc(h, (void**)&h->rhs_bg, E * 3 * np * sizeof(double));
  if (!st && !h->fflux64)
    st = dev_alloc(h, (void**)&h->fflux64, (size_t)h->g.nfaces * 5 * nf2 * sizeof(double));
  if (!st && !h->bg3) st = dev_alloc(h, (void**)&h->bg3, E * 3 * np * sizeof(double));
  if (!st && !h->bgp) st = dev_alloc(h, (void**)&h->bgp, E * 4 * np * sizeof(float));
  if (!st && !h->rhs_bg32) st = dev_alloc(h, (void**)&h->rhs_bg32, E * 3 * np * sizeof(float));
  if (st) return st;
  double* q0 = h->qtmp;
  if (q_dev == q0) return ES_DG_EINVAL;
  touch(h);
  h->bg_moving = 0;
  cudaError_t e = esdg_launch_background(h->g, h->P, h->vgeo, q_dev, h->bg, q0, h->stream);
  if (e == cudaSuccess)
    e = esdg_launch_background_vol(h->g, h->P, h->vgeo, h->bg, h->bg3, h->bgp, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (is_partition(h)) {
    // the faces of the cut planes need the neighbours' background: evaluated at the
    // first stage, after a trace exchange has brought it (resolve_background)
    h->has_bg = 1;
    h->bg_pending = 1;
    return ES_DG_OK;
  }
  e = esdg_launch_face(h->g, h->P, 0, q0, h->fgeo, h->fflux64, h->stream);
  if (e == cudaSuccess) {
    EsdgVolArgs a = vol_args(h, q0, h->rhs);
    a.vgeo = h->vgeo;
    a.fflux = h->fflux64;
    a.bg = nullptr;
    e = esdg_launch_volume(h->g, h->L, h->P, 0, 0, a, h->stream);
  }
  // momentum components: rhs[e][1..3][n] -> rhs_bg[e][0..2][n], and its FP32 copy
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(h->rhs_bg, 3 * np * sizeof(double), h->rhs + np, 5 * np * sizeof(double),
                          3 * np * sizeof(double), E, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = esdg_launch_to_f32(h->rhs_bg, h->rhs_bg32, (long long)E * 3 * np, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  h->has_bg = 1;
  h->bg_moving = 0;
  return ES_DG_OK;
}

// Set a moving background from state q_dev (device; whole meshes only): the
// state itself with its flow, its rho_bg, b_bg, p_bg and FP32 fields as for a
// background at rest, u_bg in FP32, and its full right-hand side evaluated
// once with the FP64 kernels (every component: a moving background's density
// and energy fluxes do not vanish).
int set_moving_background_dev(es_dg_t* h, const double* q_dev) {
  if (is_partition(h)) return ES_DG_EINVAL;
  const size_t E = h->g.E, np = h->g.np, nf2 = (size_t)h->g.Nq * h->g.Nq;
  int st = ensure_rhs_buffers(h);
  if (!st && !h->bg) st = dev_alloc(h, (void**)&h->bg, E * 3 * np * sizeof(double));
  if (!st && !h->fflux64)
    st = dev_alloc(h, (void**)&h->fflux64, (size_t)h->g.nfaces * 5 * nf2 * sizeof(double));
  if (!st && !h->bg3) st = dev_alloc(h, (void**)&h->bg3, E * 3 * np * sizeof(double));
  if (!st && !h->bgp) st = dev_alloc(h, (void**)&h->bgp, E * 4 * np * sizeof(float));
  if (!st && !h->bgq) st = dev_alloc(h, (void**)&h->bgq, E * 5 * np * sizeof(double));
  if (!st && !h->bgu) st = dev_alloc(h, (void**)&h->bgu, E * 3 * np * sizeof(float));
  if (!st && !h->rhs_bgm32) st = dev_alloc(h, (void**)&h->rhs_bgm32, E * 5 * np * sizeof(float));
  if (st) return st;
  if (q_dev == h->qtmp) return ES_DG_EINVAL;
  touch(h);
  h->has_bg = 0;  // until the new background is complete
  cudaError_t e = cudaMemcpyAsync(h->bgq, q_dev, E * 5 * np * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess)
    e = esdg_launch_background(h->g, h->P, h->vgeo, h->bgq, h->bg, h->qtmp, h->stream);
  if (e == cudaSuccess)
    e = esdg_launch_background_vol(h->g, h->P, h->vgeo, h->bg, h->bg3, h->bgp, h->stream);
  if (e == cudaSuccess) e = esdg_launch_background_velocity(h->g, h->bgq, h->bgu, h->stream);
  if (e == cudaSuccess) e = esdg_launch_face(h->g, h->P, 0, h->bgq, h->fgeo, h->fflux64, h->stream);
  if (e == cudaSuccess) {
    EsdgVolArgs a = vol_args(h, h->bgq, h->rhs);
    a.vgeo = h->vgeo;
    a.fflux = h->fflux64;
    a.bg = nullptr;
    a.bgq = nullptr;
    e = esdg_launch_volume(h->g, h->L, h->P, 0, 0, a, h->stream);
  }
  if (e == cudaSuccess) e = esdg_launch_to_f32(h->rhs, h->rhs_bgm32, (long long)E * 5 * np, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  h->has_bg = 1;
  h->bg_moving = 1;
  return ES_DG_OK;
}

// A mixed partition's background right-hand side, as the whole mesh evaluates it:
// the at-rest state rebuilt from the stored background, the neighbours' at-rest
// states at the cut planes from the received traces (slots 5-6).
int resolve_background(es_dg_t* h) {
  if (trace_nv(h) != 7) return ES_DG_EINVAL;  // only mixed handles carry a background
  const size_t E = h->g.E, np = h->g.np;
  double* q0 = h->qtmp;
  cudaError_t e = esdg_launch_background_state(h->g, h->P, h->vgeo, h->bg, q0, h->stream);
  if (e == cudaSuccess) {
    EsdgTraces t = traces_of(h);
    t.bgmode = 1;
    e = esdg_launch_face(h->g, h->P, 0, q0, h->fgeo, h->fflux64, h->stream, nullptr, t);
  }
  if (e == cudaSuccess) {
    EsdgVolArgs a = vol_args(h, q0, h->rhs);
    a.vgeo = h->vgeo;
    a.fflux = h->fflux64;
    a.bg = nullptr;
    e = esdg_launch_volume(h->g, h->L, h->P, 0, 0, a, h->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(h->rhs_bg, 3 * np * sizeof(double), h->rhs + np, 5 * np * sizeof(double),
                          3 * np * sizeof(double), E, cudaMemcpyDeviceToDevice, h->stream);
  if (e == cudaSuccess) e = esdg_launch_to_f32(h->rhs_bg, h->rhs_bg32, (long long)E * 3 * np, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  h->bg_pending = 0;
  touch(h);
  return ES_DG_OK;
}

}  // namespace

// The handle's status word (internal; the server reads its members' flags this
// way): 1 if a stage update since the last call produced a non-finite state or
// a non-positive density, 0 if not, -1 on a CUDA error.  Synchronous; clears it.
int esdg_take_status(es_dg_t* h) {
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && v) e = cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return v ? 1 : 0;
}

// Batch descriptor of a handle for the server's persistent kernels (not part of
// the C ABI).  Mixed-precision members must carry a background.
int esdg_member_descriptor(es_dg_t* h, double dt, EsdgMember* out, EsdgLGL* L, int* mixed) {
  if (!h || !out) return ES_DG_EINVAL;
  if (h->mixed && !h->has_bg) return ES_DG_EINVAL;
  if (h->mixed && h->bg_moving) return ES_DG_EINVAL;  // batched kernels: a background at rest
  if (is_partition(h)) return ES_DG_EINVAL;  // batched members are whole meshes
  std::memset(out, 0, sizeof(*out));
  out->g = h->g;
  out->P = h->P;
  out->a = vol_args(h, h->q, nullptr);
  out->a.dt = dt;
  out->fgeo = h->fgeo;
  out->bg = h->mixed ? h->bg : nullptr;
  if (L) *L = h->L;
  if (mixed) *mixed = h->mixed;
  return ES_DG_OK;
}

namespace {

// Same mesh, order and gravity: the geometry (coordinates, metric terms,
// Jacobian, geopotential, face normals and scalings) is identical.
bool same_geometry(const es_dg_t* a, const EsdgGrid& g, double gravity) {
  if (!a || a->g.N != g.N || a->g.warp != g.warp || a->P.g != gravity) return false;
  for (int d = 0; d < 3; d++)
    if (a->g.K[d] != g.K[d] || a->g.periodic[d] != g.periodic[d] || a->g.lo[d] != g.lo[d] ||
        a->g.hi[d] != g.hi[d] || a->g.eoff[d] != g.eoff[d] || a->g.Kg[d] != g.Kg[d])
      return false;
  return a->g.remote[0] == g.remote[0] && a->g.remote[1] == g.remote[1];
}

int create_impl(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                const es_dg_physics* physics, const es_dg_allocator* allocator, void* cuda_stream,
                const es_dg_t* geometry_of, es_dg_t** out, int x_begin = 0, int x_end = -1) {
  if (!out) return ES_DG_EINVAL;
  *out = nullptr;
  if (precision != ES_DG_FP64 && precision != ES_DG_FP32_MIXED) return ES_DG_EINVAL;
  if (allocator && (!allocator->alloc || !allocator->free)) return ES_DG_EINVAL;
  EsdgGrid g;
  int st = build_grid(mesh, N, &g, x_begin, x_end);
  if (st) return st;
  es_dg_t* h = new (std::nothrow) es_dg();
  if (!h) return ES_DG_ENOMEM;
  touch(h);
  h->g = g;
  if (esdg_lgl_build(N, &h->L)) {
    delete h;
    return ES_DG_EINVAL;
  }
  for (int i = 0; i < ESDG_MAXNQ; i++)
    for (int l = 0; l < ESDG_MAXNQ; l++) h->L.Dtf[i][l] = (float)h->L.Dt[i][l];
  if (physics) {
    h->P.gamma = physics->gamma;
    h->P.g = physics->g;
    h->P.R = physics->R;
    h->P.p0 = physics->p0;
    h->P.f0 = physics->f0;
    h->P.beta = physics->beta;
    h->P.y0 = physics->y0;
    h->P.dissipation = physics->dissipation ? 1 : 0;
    if (!(h->P.gamma > 1.0) || !(h->P.R > 0.0) || !(h->P.p0 > 0.0)) {
      delete h;
      return ES_DG_EINVAL;
    }
  } else {
    h->P = EsdgPhys{1.4, 9.81, 287.0, 1.0e5, 0.0, 0.0, 0.0, 1, 0.0, 0.0};
  }
  esdg_phys_derive(&h->P);
  {
    // gravity acts along z: a z-periodic box would make phi = g z jump across
    // the periodic faces, which the balance law does not allow
    if (g.periodic[2] && h->P.g != 0.0) {
      delete h;
      return ES_DG_EINVAL;
    }
  }
  h->mixed = (precision == ES_DG_FP32_MIXED);
  h->stream = (cudaStream_t)cuda_stream;
  if (allocator) {
    h->alloc = *allocator;
    h->has_alloc = 1;
  }
  const size_t E = g.E, np = g.np, nf2 = (size_t)g.Nq * g.Nq;
  const size_t nq = E * 5 * np;
  st = dev_alloc(h, (void**)&h->q, nq * sizeof(double));
  if (!st) st = dev_alloc(h, &h->dq, nq * (h->mixed ? sizeof(float) : sizeof(double)));
  if (!st) st = dev_alloc(h, (void**)&h->x, E * 3 * np * sizeof(double));
  if (!st) st = dev_alloc(h, (void**)&h->J, E * np * sizeof(double));
  if (!st) st = dev_alloc(h, (void**)&h->Ja, E * 9 * np * sizeof(double));
  if (!st) st = dev_alloc(h, (void**)&h->vgeo, E * ESDG_NVGEO * np * sizeof(double));
  if (!st) st = dev_alloc(h, (void**)&h->vgeo32, E * ESDG_NVGEO * np * sizeof(float));
  if (!st) st = dev_alloc(h, (void**)&h->fgeo, (size_t)g.nfaces * 5 * nf2 * sizeof(double));
  if (!st)
    st = dev_alloc(h, &h->fflux,
                   (size_t)g.nfaces * 5 * nf2 * (h->mixed ? sizeof(float) : sizeof(double)));
  if (!st) st = dev_alloc(h, (void**)&h->scratch, esdg_reduce_scratch(g) * sizeof(double));
  if (!st) st = dev_alloc(h, (void**)&h->result, 4 * sizeof(double));
  if (st) {
    es_dg_destroy(h);
    return st;
  }
  h->status = reinterpret_cast<int*>(h->result + 3);
  cudaError_t e = cudaMemsetAsync(h->result, 0, 4 * sizeof(double), h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->dq, 0, nq * (h->mixed ? sizeof(float) : sizeof(double)), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->q, 0, nq * sizeof(double), h->stream);
  if (e == cudaSuccess) {
    if (same_geometry(geometry_of, h->g, h->P.g)) {
      // device-to-device copies of an identical mesh's geometry
      const es_dg_t* o = geometry_of;
      const size_t nfg = (size_t)g.nfaces * 5 * nf2;
      const struct { void* d; const void* s; size_t b; } cp[6] = {
          {h->x, o->x, E * 3 * np * sizeof(double)},
          {h->J, o->J, E * np * sizeof(double)},
          {h->Ja, o->Ja, E * 9 * np * sizeof(double)},
          {h->vgeo, o->vgeo, E * ESDG_NVGEO * np * sizeof(double)},
          {h->vgeo32, o->vgeo32, E * ESDG_NVGEO * np * sizeof(float)},
          {h->fgeo, o->fgeo, nfg * sizeof(double)}};
      for (int k = 0; k < 6 && e == cudaSuccess; k++)
        e = cudaMemcpyAsync(cp[k].d, cp[k].s, cp[k].b, cudaMemcpyDeviceToDevice, h->stream);
    } else {
      e = esdg_launch_geometry(h->g, h->L, h->x, h->J, h->Ja, h->vgeo, h->vgeo32, h->fgeo, h->P,
                               h->stream);
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    es_dg_destroy(h);
    return cuda_status(e);
  }
  *out = h;
  return ES_DG_OK;
}

}  // namespace

namespace {
std::atomic<unsigned> g_phantom_tx{0};
}
unsigned esdg_take_phantom() { return g_phantom_tx.exchange(0u); }

// Internal (server): create a handle whose geometry is copied from `geometry_of`
// when that handle has the same mesh, order and gravity (else computed).
int esdg_create_from(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                     const es_dg_physics* physics, void* cuda_stream, const es_dg_t* geometry_of,
                     es_dg_t** out) {
  return create_impl(mesh, N, precision, physics, nullptr, cuda_stream, geometry_of, out);
}

extern "C" {

int es_dg_create(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                 const es_dg_physics* physics, const es_dg_allocator* allocator,
                 void* cuda_stream, es_dg_t** out) {
  return create_impl(mesh, N, precision, physics, allocator, cuda_stream, nullptr, out);
}

void es_dg_destroy(es_dg_t* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->pexec) cudaGraphExecDestroy(h->pexec);
  if (h->pstream) {
    cudaStreamSynchronize(h->pstream);
    cudaEventDestroy(h->ev_packed);
    cudaEventDestroy(h->ev_sent);
    cudaEventDestroy(h->ev_faced);
    cudaEventDestroy(h->ev_join);
    cudaStreamDestroy(h->pstream);
  }
  for (void* p : h->blocks) {
    if (h->has_alloc) h->alloc.free(p, h->alloc.ctx);
    else cudaFree(p);
  }
  delete h;
}

int es_dg_get_info(const es_dg_t* h, es_dg_info_t* info) {
  if (!h || !info) return ES_DG_EINVAL;
  info->N = h->g.N;
  info->Nq = h->g.Nq;
  info->np = h->g.np;
  info->nelem = h->g.E;
  info->ndof = (long long)h->g.E * h->g.np;
  info->nfaces = h->g.nfaces;
  info->device_bytes = h->bytes;
  info->precision = h->mixed ? ES_DG_FP32_MIXED : ES_DG_FP64;
  return ES_DG_OK;
}

int es_dg_set_state(es_dg_t* h, const double* q, int on_device) {
  if (!h || !q) return ES_DG_EINVAL;
  const size_t bytes = (size_t)h->g.E * 5 * h->g.np * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(h->q, q, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

int es_dg_get_state(es_dg_t* h, double* q, int on_device) {
  if (!h || !q) return ES_DG_EINVAL;
  const size_t bytes = (size_t)h->g.E * 5 * h->g.np * sizeof(double);
  cudaError_t e = cudaMemcpyAsync(q, h->q, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                            : cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

int es_dg_init_bubble(es_dg_t* h, double theta0, double amp, const double centre[3],
                      double radius) {
  return es_dg_init_bubble_profile(h, theta0, amp, centre, radius, ES_DG_BUBBLE_SMOOTH);
}

int es_dg_init_bubble_profile(es_dg_t* h, double theta0, double amp, const double centre[3],
                              double radius, int profile) {
  if (!h || !centre || !(theta0 > 0.0) || !(radius > 0.0)) return ES_DG_EINVAL;
  if (profile != ES_DG_BUBBLE_SMOOTH && profile != ES_DG_BUBBLE_SHARP) return ES_DG_EINVAL;
  const int sharp = profile == ES_DG_BUBBLE_SHARP;
  cudaError_t e;
  if (h->mixed) {
    // the unperturbed isentropic atmosphere is the mixed path's background
    int st = ensure_rhs_buffers(h);
    if (st) return st;
    e = esdg_launch_bubble(h->g, h->P, h->x, theta0, 0.0, centre, radius, sharp, h->q,
                           h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemcpyAsync(h->rhs, h->q, (size_t)h->g.E * 5 * h->g.np * sizeof(double),
                        cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    st = set_background_dev(h, h->rhs);
    if (st) return st;
  }
  e = esdg_launch_bubble(h->g, h->P, h->x, theta0, amp, centre, radius, sharp, h->q, h->stream);
  return cuda_status(e);
}

int es_dg_init_channel(es_dg_t* h) {
  return es_dg_init_channel_ex(h, 1.0, ES_DG_BACKGROUND_REST);
}

int es_dg_init_channel_ex(es_dg_t* h, double amp, int background) {
  if (!h || !std::isfinite(amp)) return ES_DG_EINVAL;
  if (background != ES_DG_BACKGROUND_REST && background != ES_DG_BACKGROUND_JET)
    return ES_DG_EINVAL;
  if (h->P.f0 == 0.0 && h->P.beta == 0.0) return ES_DG_EINVAL;  // geostrophic balance needs f
  if (h->mixed && background == ES_DG_BACKGROUND_JET && is_partition(h)) return ES_DG_EINVAL;
  cudaError_t e;
  if (h->mixed && background == ES_DG_BACKGROUND_JET) {
    // the balanced jet alone (no perturbation), carried with its velocity
    int st = ensure_rhs_buffers(h);
    if (st) return st;
    e = esdg_launch_channel(h->g, h->P, h->x, h->q, 0.0, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    st = set_moving_background_dev(h, h->q);
    if (st) return st;
  }
  e = esdg_launch_channel(h->g, h->P, h->x, h->q, amp, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (h->mixed && background == ES_DG_BACKGROUND_REST)
    return set_background_dev(h, h->q);  // the state at rest
  return ES_DG_OK;
}

int es_dg_set_background(es_dg_t* h, const double* q_bg, int on_device) {
  if (!h || !q_bg) return ES_DG_EINVAL;
  if (!h->mixed) return ES_DG_OK;  // the FP64 path needs no background
  const size_t bytes = (size_t)h->g.E * 5 * h->g.np * sizeof(double);
  int st = ensure_rhs_buffers(h);
  if (st) return st;
  // stage the input in the rhs buffer (the background's own evaluation uses qtmp)
  cudaError_t e = cudaMemcpyAsync(h->rhs, q_bg, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  st = set_background_dev(h, h->rhs);
  if (!st && !on_device) st = cuda_status(cudaStreamSynchronize(h->stream));
  return st;
}

int es_dg_set_moving_background(es_dg_t* h, const double* q_bg, int on_device) {
  if (!h || !q_bg) return ES_DG_EINVAL;
  if (!h->mixed) return ES_DG_OK;  // the FP64 path needs no background
  if (is_partition(h)) return ES_DG_EINVAL;
  const size_t bytes = (size_t)h->g.E * 5 * h->g.np * sizeof(double);
  int st = ensure_rhs_buffers(h);
  if (st) return st;
  cudaError_t e = cudaMemcpyAsync(h->rhs, q_bg, bytes, on_device ? cudaMemcpyDeviceToDevice
                                                                 : cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  st = set_moving_background_dev(h, h->rhs);
  if (!st && !on_device) st = cuda_status(cudaStreamSynchronize(h->stream));
  return st;
}

int es_dg_clear_background(es_dg_t* h) {
  if (!h) return ES_DG_EINVAL;
  touch(h);
  h->has_bg = 0;
  h->bg_pending = 0;
  h->bg_moving = 0;
  return ES_DG_OK;
}

int es_dg_rhs(es_dg_t* h, const double* q, double* rhs, int on_device) {
  if (!h || !q || !rhs) return ES_DG_EINVAL;
  const size_t bytes = (size_t)h->g.E * 5 * h->g.np * sizeof(double);
  const double* qin = q;
  double* rout = rhs;
  if (!on_device) {
    int st = ensure_rhs_buffers(h);
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(h->qtmp, q, bytes, cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return cuda_status(e);
    qin = h->qtmp;
    rout = h->rhs;
  }
  int st = launch_stage(h, qin, 0, rout, 0.0, 0.0, 0.0);
  if (st) return st;
  if (!on_device) {
    cudaError_t e = cudaMemcpyAsync(rhs, h->rhs, bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return cuda_status(e);
  }
  return ES_DG_OK;
}

int es_dg_cfl_dt(es_dg_t* h, double C, double* dt) {
  if (!h || !dt || !(C > 0.0)) return ES_DG_EINVAL;
  cudaError_t e = esdg_launch_cfl(h->g, h->L, h->P, h->q, h->x, h->J, h->Ja, h->scratch, h->result,
                                  h->stream);
  double r = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, h->result, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_status(e);
  if (!(r > 0.0) || r != r) return ES_DG_ENAN;
  *dt = C * (h->L.xi[1] - h->L.xi[0]) * r;
  return ES_DG_OK;
}

int es_dg_step(es_dg_t* h, double dt, int nsteps) {
  if (!h || nsteps < 0 || !(dt > 0.0)) return ES_DG_EINVAL;
  if (is_partition(h)) return ES_DG_EINVAL;  // stages need the trace exchange
  for (int n = 0; n < nsteps; n++)
    for (int s = 0; s < 5; s++) {
      int st = launch_stage(h, h->q, 1, nullptr, kRkA[s], kRkB[s], dt);
      if (st) return st;
    }
  return ES_DG_OK;
}

void es_dg_debug_inject_wait_timeout(void) { g_phantom_tx.store(16u); }

int es_dg_sync(es_dg_t* h) {
  if (!h) return ES_DG_EINVAL;
  const int st = cuda_status(cudaStreamSynchronize(h->stream));
  if (st != ES_DG_OK) return st;
  const int t64 = esdg_volume_f64_take_timeout(), t32 = esdg_volume_mixed_take_timeout();
  if (t64 < 0 || t32 < 0) return ES_DG_ECUDA;
  if (t64 || t32) return ES_DG_ETIMEOUT;
  const int bad = esdg_take_status(h);
  if (bad < 0) return ES_DG_ECUDA;
  return bad ? ES_DG_ENAN : ES_DG_OK;
}

int es_dg_integrals(es_dg_t* h, double out[3]) {
  if (!h || !out) return ES_DG_EINVAL;
  cudaError_t e = esdg_launch_integrals(h->g, h->L, h->P, h->q, h->J, h->x, h->scratch, h->result,
                                        h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->result, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

int es_dg_geometry(es_dg_t* h, double* x, double* J, double* Ja, int on_device) {
  if (!h) return ES_DG_EINVAL;
  const size_t E = h->g.E, np = h->g.np;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaSuccess;
  if (x) e = cudaMemcpyAsync(x, h->x, E * 3 * np * sizeof(double), k, h->stream);
  if (e == cudaSuccess && J) e = cudaMemcpyAsync(J, h->J, E * np * sizeof(double), k, h->stream);
  if (e == cudaSuccess && Ja) e = cudaMemcpyAsync(Ja, h->Ja, E * 9 * np * sizeof(double), k, h->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
  return cuda_status(e);
}

int es_dg_launch(es_dg_t* h, int which, int stage, double dt) {
  if (!h || stage < 0 || stage > 4) return ES_DG_EINVAL;
  if (!traces_ready(h)) return ES_DG_EINVAL;
  // the faces that need no trace may run before the traces arrive; everything
  // else first completes a pending background (which reads them)
  if (h->bg_pending && which != 3) {
    const int st = resolve_background(h);
    if (st) return st;
  }
  if (which == 0) return launch_faces(h, h->q, FACES_ALL);
  if (which == 3) return launch_faces(h, h->q, FACES_INTERIOR);
  if (which == 4) return launch_faces(h, h->q, FACES_CUT);
  if (which == 1) {
    int st = ensure_rhs_buffers(h);
    if (st) return st;
    EsdgVolArgs a = vol_args(h, h->q, h->rhs);
    return cuda_status(esdg_launch_volume(h->g, h->L, h->P, h->mixed, 0, a, h->stream));
  }
  if (which == 2) {
    EsdgVolArgs a = vol_args(h, h->q, nullptr);
    a.rkA = kRkA[stage];
    a.rkB = kRkB[stage];
    a.dt = dt;
    return cuda_status(esdg_launch_volume(h->g, h->L, h->P, h->mixed, 1, a, h->stream));
  }
  return ES_DG_EINVAL;
}

// ---- domain decomposition along x -----------------------------------------

int es_dg_create_partition(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                           const es_dg_physics* physics, int x_begin, int x_end,
                           const es_dg_allocator* allocator, void* cuda_stream, es_dg_t** out) {
  if (x_end < 0) return ES_DG_EINVAL;
  return create_impl(mesh, N, precision, physics, allocator, cuda_stream, nullptr, out, x_begin,
                     x_end);
}

int es_dg_partition_info(const es_dg_t* h, int* x_begin, int* x_end, int remote[2],
                         long long* trace_len) {
  if (!h) return ES_DG_EINVAL;
  if (x_begin) *x_begin = h->g.eoff[0];
  if (x_end) *x_end = h->g.eoff[0] + h->g.K[0];
  if (remote) {
    remote[0] = h->g.remote[0];
    remote[1] = h->g.remote[1];
  }
  if (trace_len) *trace_len = (long long)trace_doubles(h);
  return ES_DG_OK;
}

int es_dg_set_traces(es_dg_t* h, double* send_lo, double* send_hi, double* recv_lo,
                     double* recv_hi) {
  if (!h) return ES_DG_EINVAL;
  if (h->g.remote[0] && (!send_lo || !recv_lo)) return ES_DG_EINVAL;
  if (h->g.remote[1] && (!send_hi || !recv_hi)) return ES_DG_EINVAL;
  for (const void* p : {(const void*)send_lo, (const void*)send_hi, (const void*)recv_lo,
                        (const void*)recv_hi})
    if (reinterpret_cast<uintptr_t>(p) % sizeof(double)) return ES_DG_EINVAL;
  touch(h);
  h->tr_send[0] = h->g.remote[0] ? send_lo : nullptr;
  h->tr_send[1] = h->g.remote[1] ? send_hi : nullptr;
  h->tr_recv[0] = h->g.remote[0] ? recv_lo : nullptr;
  h->tr_recv[1] = h->g.remote[1] ? recv_hi : nullptr;
  return ES_DG_OK;
}

int es_dg_pack_traces(es_dg_t* h, int what) {
  if (!h) return ES_DG_EINVAL;
  for (int s = 0; s < 2; s++)
    if (h->g.remote[s] && !h->tr_send[s]) return ES_DG_EINVAL;
  if (what == ES_DG_TRACE_STATE)
    return cuda_status(esdg_launch_trace_pack(h->g, h->q, (h->mixed && h->has_bg) ? h->bg : nullptr,
                                              trace_nv(h), h->tr_send[0], h->tr_send[1],
                                              h->stream));
  if (what == ES_DG_TRACE_GEOMETRY) {
    // the high plane's face geometry (its "-" element is this partition's)
    if (!h->g.remote[1]) return ES_DG_OK;
    const size_t nf2 = (size_t)h->g.Nq * h->g.Nq, plane = (size_t)h->g.K[1] * h->g.K[2];
    const double* src = h->fgeo + ((size_t)h->g.face_off[0] + (size_t)h->g.K[0] * plane) * 5 * nf2;
    return cuda_status(cudaMemcpyAsync(h->tr_send[1], src, plane * 5 * nf2 * sizeof(double),
                                       cudaMemcpyDeviceToDevice, h->stream));
  }
  return ES_DG_EINVAL;
}

int es_dg_accept_geometry_trace(es_dg_t* h) {
  if (!h) return ES_DG_EINVAL;
  if (!h->g.remote[0]) return ES_DG_OK;
  if (!h->tr_recv[0]) return ES_DG_EINVAL;
  const size_t nf2 = (size_t)h->g.Nq * h->g.Nq, plane = (size_t)h->g.K[1] * h->g.K[2];
  double* dst = h->fgeo + (size_t)h->g.face_off[0] * 5 * nf2;  // plane 0 of direction x
  return cuda_status(cudaMemcpyAsync(dst, h->tr_recv[0], plane * 5 * nf2 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->stream));
}

namespace {

// Partitions in x order on one stream with their traces set; returns the
// neighbour across each remote plane through lo_of / hi_of.
int check_partitions(es_dg_t* const* parts, int P, std::vector<int>& lo_of, std::vector<int>& hi_of) {
  if (!parts || P < 1) return ES_DG_EINVAL;
  lo_of.assign(P, -1);
  hi_of.assign(P, -1);
  for (int p = 0; p < P; p++) {
    const es_dg_t* h = parts[p];
    if (!h || h->stream != parts[0]->stream || h->mixed != parts[0]->mixed ||
        h->g.N != parts[0]->g.N)
      return ES_DG_EINVAL;
    for (int d = 0; d < 3; d++)
      if (h->g.Kg[d] != parts[0]->g.Kg[d]) return ES_DG_EINVAL;
    for (int d = 1; d < 3; d++)
      if (h->g.K[d] != parts[0]->g.K[d]) return ES_DG_EINVAL;
    const int next = (p + 1 < P) ? p + 1 : 0;
    const bool last = (p + 1 == P);
    // contiguous cover of the parent's x layers, in order
    if (!last && h->g.eoff[0] + h->g.K[0] != parts[next]->g.eoff[0]) return ES_DG_EINVAL;
    if (p == 0 && h->g.eoff[0] != 0) return ES_DG_EINVAL;
    if (last && h->g.eoff[0] + h->g.K[0] != h->g.Kg[0]) return ES_DG_EINVAL;
    if (h->g.remote[1]) {
      if (!parts[next]->g.remote[0] || (last && P < 2)) return ES_DG_EINVAL;
      hi_of[p] = next;
      lo_of[next] = p;
    }
    if (!traces_ready(h)) return ES_DG_EINVAL;
    for (int s = 0; s < 2; s++)
      if (h->g.remote[s] && !h->tr_send[s]) return ES_DG_EINVAL;
  }
  for (int p = 0; p < P; p++)
    if (parts[p]->g.remote[0] && lo_of[p] < 0) return ES_DG_EINVAL;
  return ES_DG_OK;
}

// copy every partition's outgoing trace into its neighbour's receive buffer
int exchange_traces(es_dg_t* const* parts, int P, const std::vector<int>& hi_of, bool geometry_only) {
  for (int p = 0; p < P; p++) {
    const es_dg_t* h = parts[p];
    const size_t bytes = trace_doubles(h) * sizeof(double);
    const int q = hi_of[p];
    if (q < 0) continue;
    // p's high plane is q's low plane
    cudaError_t e = cudaMemcpyAsync(parts[q]->tr_recv[0], h->tr_send[1], bytes,
                                    cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && !geometry_only)
      e = cudaMemcpyAsync(h->tr_recv[1], parts[q]->tr_send[0], bytes, cudaMemcpyDeviceToDevice,
                          h->stream);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return ES_DG_OK;
}

}  // namespace

int es_dg_partitions_connect(es_dg_t* const* parts, int P) {
  std::vector<int> lo_of, hi_of;
  int st = check_partitions(parts, P, lo_of, hi_of);
  for (int p = 0; p < P && !st; p++) st = es_dg_pack_traces(parts[p], ES_DG_TRACE_GEOMETRY);
  if (!st) st = exchange_traces(parts, P, hi_of, true);
  for (int p = 0; p < P && !st; p++) st = es_dg_accept_geometry_trace(parts[p]);
  if (!st) st = cuda_status(cudaStreamSynchronize(parts[0]->stream));
  return st;
}

int es_dg_partitions_exchange(es_dg_t* const* parts, int P) {
  std::vector<int> lo_of, hi_of;
  int st = check_partitions(parts, P, lo_of, hi_of);
  for (int p = 0; p < P && !st; p++) st = es_dg_pack_traces(parts[p], ES_DG_TRACE_STATE);
  if (!st) st = exchange_traces(parts, P, hi_of, false);
  return st;
}

namespace {

int ensure_part_streams(es_dg_t* h) {
  if (h->pstream) return ES_DG_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->pstream, cudaStreamNonBlocking);
  cudaEvent_t* evs[4] = {&h->ev_packed, &h->ev_sent, &h->ev_faced, &h->ev_join};
  for (int k = 0; k < 4 && e == cudaSuccess; k++)
    e = cudaEventCreateWithFlags(evs[k], cudaEventDisableTiming);
  return cuda_status(e);
}

// One LSRK step of all partitions, each on its own stream (h->stream is the
// partition's pstream meanwhile), ordered by events instead of one stream:
//   A1  every partition packs its traces (after its previous stage);
//   A2  partition p copies the pair of traces across its high plane into the
//       receive buffers of p and q = hi_of[p], after q's pack and after q's
//       previous face pass (which read the buffer being overwritten);
//   B   each partition runs its faces once its low neighbour's copies have
//       landed, then its volume kernel with the stage update.
// The host issues the phases in this order for every stage, so each wait
// names an event already recorded for this stage (A1 -> A2 -> B) or the
// previous one (B -> A2): the dependency graph has no cycle.  Partitions'
// kernels overlap where their dependencies allow (one slab's volume kernel
// with a neighbour's faces and copies) instead of running one after another.
// captured: the step is being captured into a graph whose launches follow one
// another, so its first stage needs (and may name) no event of the step before.
int issue_partition_step(es_dg_t* const* parts, int P, const std::vector<int>& lo_of,
                         const std::vector<int>& hi_of, double dt, bool captured) {
  for (int s = 0; s < 5; s++) {
    for (int p = 0; p < P; p++) {
      int st = es_dg_pack_traces(parts[p], ES_DG_TRACE_STATE);
      if (st) return st;
      if (cudaEventRecord(parts[p]->ev_packed, parts[p]->stream) != cudaSuccess) return ES_DG_ECUDA;
    }
    for (int p = 0; p < P; p++) {
      es_dg_t* h = parts[p];
      const int q = hi_of[p];
      if (q < 0) continue;
      cudaError_t e = cudaStreamWaitEvent(h->stream, parts[q]->ev_packed, 0);
      if (e == cudaSuccess && q != p && !(captured && s == 0))
        e = cudaStreamWaitEvent(h->stream, parts[q]->ev_faced, 0);
      const size_t bytes = trace_doubles(h) * sizeof(double);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(parts[q]->tr_recv[0], h->tr_send[1], bytes, cudaMemcpyDeviceToDevice,
                            h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->tr_recv[1], parts[q]->tr_send[0], bytes, cudaMemcpyDeviceToDevice,
                            h->stream);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_sent, h->stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
    for (int p = 0; p < P; p++) {
      es_dg_t* h = parts[p];
      // one face launch once the traces are in: on one GPU the copies are short,
      // and splitting off the faces that need no trace (as a process per slab
      // does, es_dg_launch 3 and 4) costs more launches than it overlaps
      if (lo_of[p] >= 0 && lo_of[p] != p &&
          cudaStreamWaitEvent(h->stream, parts[lo_of[p]]->ev_sent, 0) != cudaSuccess)
        return ES_DG_ECUDA;
      int st = ES_DG_OK;
      if (h->bg_pending) {
        st = resolve_background(h);
        if (st) return st;
      }
      st = launch_faces(h, h->q, FACES_ALL);
      if (st) return st;
      cudaError_t e = cudaEventRecord(h->ev_faced, h->stream);
      if (e != cudaSuccess) return cuda_status(e);
      EsdgVolArgs a = vol_args(h, h->q, nullptr);
      a.rkA = kRkA[s];
      a.rkB = kRkB[s];
      a.dt = dt;
      e = esdg_launch_volume(h->g, h->L, h->P, h->mixed, 1, a, h->stream);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  return ES_DG_OK;
}

}  // namespace

namespace {

// The captured step of parts (led by parts[0]) is valid for this call: same time
// step, same partitions, none of them reconfigured since, no background pending.
bool step_graph_valid(es_dg_t* const* parts, int P, double dt) {
  const es_dg_t* h0 = parts[0];
  if (!h0->pexec || h0->pexec_dt != dt || (int)h0->pexec_parts.size() != P) return false;
  for (int p = 0; p < P; p++)
    if (h0->pexec_parts[p] != parts[p] || h0->pexec_gens[p] != parts[p]->gen ||
        parts[p]->bg_pending)
      return false;
  return true;
}

// Capture one LSRK step of parts on the first partition's stream (every other
// partition stream joined into the capture) and keep it in parts[0].
int capture_step_graph(es_dg_t* const* parts, int P, const std::vector<int>& lo_of,
                       const std::vector<int>& hi_of, double dt) {
  es_dg_t* h0 = parts[0];
  cudaStream_t o = h0->pstream;
  if (h0->pexec) {
    cudaGraphExecDestroy(h0->pexec);
    h0->pexec = nullptr;
  }
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaEventRecord(h0->ev_join, o);
  for (int p = 1; p < P && e == cudaSuccess; p++)
    e = cudaStreamWaitEvent(parts[p]->stream, h0->ev_join, 0);
  int st = e == cudaSuccess ? issue_partition_step(parts, P, lo_of, hi_of, dt, true) : ES_DG_ECUDA;
  for (int p = 1; p < P && !st; p++)
    if (cudaEventRecord(parts[p]->ev_join, parts[p]->stream) != cudaSuccess ||
        cudaStreamWaitEvent(o, parts[p]->ev_join, 0) != cudaSuccess)
      st = ES_DG_ECUDA;
  e = cudaStreamEndCapture(o, &gr);
  if (!st && e != cudaSuccess) st = cuda_status(e);
  if (!st) st = cuda_status(cudaGraphInstantiate(&h0->pexec, gr, 0));
  if (gr) cudaGraphDestroy(gr);
  if (st) {
    cudaGetLastError();
    h0->pexec = nullptr;
    return st;
  }
  h0->pexec_dt = dt;
  h0->pexec_parts.assign(parts, parts + P);
  h0->pexec_gens.resize(P);
  for (int p = 0; p < P; p++) h0->pexec_gens[p] = parts[p]->gen;
  return ES_DG_OK;
}

}  // namespace

int es_dg_partitions_step(es_dg_t* const* parts, int P, double dt, int nsteps) {
  if (nsteps < 0 || !(dt > 0.0)) return ES_DG_EINVAL;
  std::vector<int> lo_of, hi_of;
  int st = check_partitions(parts, P, lo_of, hi_of);
  if (st || nsteps == 0) return st;
  for (int p = 0; p < P && !st; p++) st = ensure_part_streams(parts[p]);
  if (st) return st;
  cudaStream_t user = parts[0]->stream;
  es_dg_t* h0 = parts[0];
  cudaStream_t o = h0->pstream;
  // fork: every partition stream after the work already queued on the caller's stream
  cudaError_t e = cudaEventRecord(h0->ev_join, user);
  for (int p = 0; p < P && e == cudaSuccess; p++) e = cudaStreamWaitEvent(parts[p]->pstream, h0->ev_join, 0);
  if (e != cudaSuccess) return cuda_status(e);
  for (int p = 0; p < P; p++) parts[p]->stream = parts[p]->pstream;
  // Steps replay the captured step graph of these partitions.  Without a valid
  // one, the first step runs as issued (it resolves a mixed partition's
  // background and configures each kernel once, outside any capture) and the
  // step is captured for the others and for later calls.
  int n = 0;
  if (!step_graph_valid(parts, P, dt)) {
    st = issue_partition_step(parts, P, lo_of, hi_of, dt, false);
    n = 1;
    // the graph runs on the first partition's stream: after every partition's first step
    for (int p = 1; p < P && !st; p++)
      if (cudaEventRecord(parts[p]->ev_join, parts[p]->stream) != cudaSuccess ||
          cudaStreamWaitEvent(o, parts[p]->ev_join, 0) != cudaSuccess)
        st = ES_DG_ECUDA;
    if (!st && capture_step_graph(parts, P, lo_of, hi_of, dt) != ES_DG_OK) {
      // no graph: issue the remaining steps directly
      for (; n < nsteps && !st; n++) st = issue_partition_step(parts, P, lo_of, hi_of, dt, false);
    }
  }
  for (; n < nsteps && !st; n++) st = cuda_status(cudaGraphLaunch(h0->pexec, o));
  // join: the caller's stream after every partition stream.  The ordering events
  // are recorded again outside any capture, so that none names a node of the
  // captured graph when the next call waits on it.
  for (int p = 0; p < P; p++) {
    es_dg_t* h = parts[p];
    h->stream = user;
    cudaError_t ej = cudaEventRecord(h->ev_packed, h->pstream);
    if (ej == cudaSuccess) ej = cudaEventRecord(h->ev_sent, h->pstream);
    if (ej == cudaSuccess) ej = cudaEventRecord(h->ev_faced, h->pstream);
    if (ej == cudaSuccess) ej = cudaEventRecord(h->ev_join, h->pstream);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(user, h->ev_join, 0);
    if (ej != cudaSuccess && !st) st = cuda_status(ej);
  }
  return st;
}

const char* es_dg_strerror(int status) {
  switch (status) {
    case ES_DG_OK: return "ok";
    case ES_DG_PENDING: return "pending";
    case ES_DG_EINVAL: return "invalid argument";
    case ES_DG_ENOMEM: return "out of device memory or over budget";
    case ES_DG_ECUDA: return "CUDA error";
    case ES_DG_ENAN: return "non-finite or non-physical state";
    case ES_DG_ETIMEOUT: return "bounded device wait timed out";
    case ES_DG_EBUSY: return "queue full";
    case ES_DG_ECANCELED: return "cancelled";
    default: return "unknown status";
  }
}

}  // extern "C"
