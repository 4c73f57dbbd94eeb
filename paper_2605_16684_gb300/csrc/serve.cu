// serve.cu -- batched ensemble and continuous-batching server (es_dg_server_*,
// es_dg_batch_submit / es_dg_batch_poll).
//
// Resident solves ("members") are ordinary es_dg handles.  Members with the
// same polynomial order and precision form a group; every LSRK stage launches,
// per group, one persistent interface-flux kernel and one persistent volume
// kernel that stride over device work tables of (member, tile) entries.  One
// whole LSRK step (5 stages x groups x 2 launches) is captured once as a CUDA
// graph and replayed; admitting or retiring a member rewrites the tables and
// the member descriptors in device memory, not the graph (the tile counts live
// in device memory).  A new group or a table that outgrows its capacity
// re-captures the graph.  Per group an autotuner picks the tile shape
// (elements per CTA) and the persistent grid size by timing real launches on
// the resident members with zero RK weights (state untouched).
//
// Admission is first-come-first-served by HBM footprint: a request waits until
// its estimated bytes fit under the server's budget and a slot is free.  A
// scheduler thread admits, steps, and retires; submit and poll are thread-safe.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/es_dg.h"
#include "esdg_internal.cuh"

// provided by api.cu for the server (internal, not part of the C ABI)
int esdg_member_descriptor(es_dg_t* h, double dt, EsdgMember* out, EsdgLGL* L, int* mixed);
int esdg_create_from(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                     const es_dg_physics* physics, void* cuda_stream, const es_dg_t* geometry_of,
                     es_dg_t** out);

namespace {

const double kA[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                      -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kB[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                      1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                      2277821191437.0 / 14882151754819.0};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Member {
  uint64_t ticket = 0;
  es_dg_request req{};
  es_dg_t* h = nullptr;
  int N = 0, mixed = 0;
  double dt = 0.0;
  int steps_done = 0;
  double t_submit = 0, t_admit = 0, t_finish = 0;
  size_t bytes = 0;
  long long ndof = 0;
  int failed = 0;  // ES_DG_ENAN once its state was flagged: finished early, alone
};

struct Group {
  int N = 0, mixed = 0;
  int variant = -1, grid_vol = 0, grid_face = 0;
  EsdgLGL L{};
  int2* d_vt = nullptr;  // volume tiles
  int2* d_ft = nullptr;  // face tiles
  int* d_n = nullptr;    // [2]: volume tiles, face tiles
  int cap_v = 0, cap_f = 0;
  std::vector<int2> vt, ft;
};

struct Result {
  es_dg_result r{};
};

// es_dg_server_warmup's request to the scheduler thread (lives on the caller's
// stack until done is set)
struct WarmJob {
  std::vector<int> orders;
  int mixed = 0;
  int status = 0;
  bool done = false;
};

size_t estimate_bytes(const es_dg_request& q) {
  const size_t Nq = q.N + 1, np = Nq * Nq * Nq, E = (size_t)q.kx * q.ky * q.kz;
  const size_t nf = 3 * (E + (size_t)q.kx * q.ky + (size_t)q.ky * q.kz + (size_t)q.kx * q.kz);
  size_t per_node = 40 + (q.precision == ES_DG_FP32_MIXED ? 20 : 40) + 24 + 8 + 72 + 88 + 44;
  size_t per_face_node = 40 + (q.precision == ES_DG_FP32_MIXED ? 20 + 40 : 40);
  if (q.precision == ES_DG_FP32_MIXED) per_node += 24 + 24 + 40 + 40;  // background, rhs, staging
  return E * np * per_node + nf * Nq * Nq * per_face_node + E * 24 + (1 << 16);
}

}  // namespace

struct es_dg_server {
  size_t budget = 0, used = 0;
  int max_slots = 0;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::unique_ptr<Member>> pending;
  std::vector<std::unique_ptr<Member>> active;
  std::map<uint64_t, Result> done;
  std::map<uint64_t, int> cancelled;
  std::deque<WarmJob*> warm_jobs;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // batch state (worker thread only)
  std::vector<Group> groups;
  EsdgMember* d_members = nullptr;
  int cap_members = 0;
  std::vector<EsdgMember> h_members;
  // per-member status words of the descriptor table (set by a stage update whose
  // state is not finite or has a non-positive density), polled every few steps
  int* d_flags = nullptr;
  int* h_flags = nullptr;  // pinned
  int n_table = 0;         // members in the uploaded table (the first n_table of active)
  int steps_since_poll = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  int use_graph = 1;
  int force_variant = -1;  // ES_DG_BATCH_VARIANT: skip the autotuner (tests)
  std::map<long long, std::pair<int, int>> tuned;  // (N, mixed) -> (variant, grid mult)
  // statistics
  es_dg_server_stats_t st{};
  double t0 = 0;
  int last_error = 0;
  bool own_stream = false;
  char msg[96] = {0};
};

namespace {

int cuda_fail(es_dg_server* s, cudaError_t e, const char* where) {
  std::snprintf(s->msg, sizeof(s->msg), "%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? ES_DG_ENOMEM : ES_DG_ECUDA;
}

int group_index(es_dg_server* s, int N, int mixed) {
  for (size_t i = 0; i < s->groups.size(); i++)
    if (s->groups[i].N == N && s->groups[i].mixed == mixed) return (int)i;
  return -1;
}

int vol_epb(const Group& g, int variant) {
  return g.mixed ? esdg_volume_batch_mixed(1, g.N, variant, nullptr, nullptr, nullptr, 0, g.L, 0, 0, 0)
                 : esdg_volume_batch_f64(1, g.N, variant, nullptr, nullptr, nullptr, 0, g.L, 0, 0, 0);
}
int vol_occ(const Group& g, int variant) {
  return g.mixed ? esdg_volume_batch_mixed(2, g.N, variant, nullptr, nullptr, nullptr, 0, g.L, 0, 0, 0)
                 : esdg_volume_batch_f64(2, g.N, variant, nullptr, nullptr, nullptr, 0, g.L, 0, 0, 0);
}
int vol_launch(es_dg_server* s, const Group& g, double A, double B) {
  const int r = g.mixed ? esdg_volume_batch_mixed(0, g.N, g.variant, s->d_members, g.d_vt, g.d_n,
                                                  g.grid_vol, g.L, A, B, s->stream)
                        : esdg_volume_batch_f64(0, g.N, g.variant, s->d_members, g.d_vt, g.d_n,
                                                g.grid_vol, g.L, A, B, s->stream);
  return r == 0 ? ES_DG_OK : cuda_fail(s, cudaGetLastError(), "volume batch launch");
}
int face_launch(es_dg_server* s, const Group& g) {
  cudaError_t e = esdg_launch_face_batch(g.N, g.mixed, g.mixed, s->d_members, g.d_ft, g.d_n + 1,
                                         g.grid_face, s->stream);
  return e == cudaSuccess ? ES_DG_OK : cuda_fail(s, e, "face batch launch");
}

void build_tiles(es_dg_server* s, Group& g, int variant) {
  const int epb = vol_epb(g, variant);
  g.vt.clear();
  g.ft.clear();
  for (size_t m = 0; m < s->active.size(); m++) {
    const Member& mb = *s->active[m];
    if (mb.N != g.N || mb.mixed != g.mixed) continue;
    const EsdgGrid& gr = s->h_members[m].g;
    for (int e0 = 0; e0 < gr.E; e0 += epb) g.vt.push_back(make_int2((int)m, e0));
    const long long nfn = gr.nfaces * gr.Nq * gr.Nq;
    for (long long f0 = 0; f0 < nfn; f0 += 256) g.ft.push_back(make_int2((int)m, (int)f0));
  }
}

// copy tables and descriptors to the device (synchronous on the stream)
int upload(es_dg_server* s) {
  const int nm = (int)s->active.size();
  if (nm > s->cap_members) {
    if (s->d_members) cudaFree(s->d_members);
    if (s->d_flags) cudaFree(s->d_flags);
    if (s->h_flags) cudaFreeHost(s->h_flags);
    s->d_flags = nullptr;
    s->h_flags = nullptr;
    s->cap_members = std::max(nm, 2 * s->cap_members);
    if (cudaMalloc(&s->d_members, sizeof(EsdgMember) * s->cap_members) != cudaSuccess ||
        cudaMalloc(&s->d_flags, sizeof(int) * s->cap_members) != cudaSuccess ||
        cudaMallocHost(&s->h_flags, sizeof(int) * s->cap_members) != cudaSuccess) {
      cudaGetLastError();
      if (s->d_members) cudaFree(s->d_members);
      if (s->d_flags) cudaFree(s->d_flags);
      s->d_members = nullptr;
      s->d_flags = nullptr;
      s->h_flags = nullptr;
      s->cap_members = 0;
      return ES_DG_ENOMEM;
    }
    s->graph_valid = false;
  }
  for (int m = 0; m < nm; m++) s->h_members[m].a.status = s->d_flags + m;
  s->n_table = nm;
  if (nm) {
    cudaError_t e = cudaMemcpyAsync(s->d_members, s->h_members.data(), sizeof(EsdgMember) * nm,
                                    cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_flags, 0, sizeof(int) * nm, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "member upload");
  }
  for (Group& g : s->groups) {
    const int nv = (int)g.vt.size(), nf = (int)g.ft.size();
    if (nv > g.cap_v || nf > g.cap_f || !g.d_n) {
      if (g.d_vt) cudaFree(g.d_vt);
      if (g.d_ft) cudaFree(g.d_ft);
      if (g.d_n) cudaFree(g.d_n);
      g.cap_v = std::max(nv, 2 * g.cap_v) + 1;
      g.cap_f = std::max(nf, 2 * g.cap_f) + 1;
      if (cudaMalloc(&g.d_vt, sizeof(int2) * g.cap_v) != cudaSuccess ||
          cudaMalloc(&g.d_ft, sizeof(int2) * g.cap_f) != cudaSuccess ||
          cudaMalloc(&g.d_n, sizeof(int) * 2) != cudaSuccess) {
        cudaGetLastError();
        return ES_DG_ENOMEM;
      }
      s->graph_valid = false;
    }
    const int n2[2] = {nv, nf};
    if ((nv && cudaMemcpyAsync(g.d_vt, g.vt.data(), sizeof(int2) * nv, cudaMemcpyHostToDevice,
                               s->stream) != cudaSuccess) ||
        (nf && cudaMemcpyAsync(g.d_ft, g.ft.data(), sizeof(int2) * nf, cudaMemcpyHostToDevice,
                               s->stream) != cudaSuccess) ||
        cudaMemcpyAsync(g.d_n, n2, sizeof(n2), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      return cuda_fail(s, cudaGetLastError(), "table upload");
  }
  // the host vectors are reused on the next change: wait for the copies
  cudaError_t e = cudaStreamSynchronize(s->stream);
  return e == cudaSuccess ? ES_DG_OK : cuda_fail(s, e, "table upload sync");
}

// Autotune one group: every tile shape x grid multiplier, timed on the current
// members with zero RK weights (B = 0 leaves the state unchanged; dq is
// rewritten at the next stage 0 anyway).
// tuning results shared by the servers of this process: (device, N, mixed) -> (variant, grid multiplier)
std::mutex g_tuned_mu;
std::map<long long, std::pair<int, int>> g_tuned;

int autotune(es_dg_server* s, Group& g) {
  const int nvar = g.mixed ? esdg_volume_batch_variants_mixed(g.N) : esdg_volume_batch_variants_f64(g.N);
  if (s->force_variant >= 0) {
    g.variant = s->force_variant < nvar ? s->force_variant : nvar - 1;
    g.grid_vol = s->sms * vol_occ(g, g.variant);
    s->graph_valid = false;
    return ES_DG_OK;
  }
  const long long key = g.N * 2 + g.mixed;
  const long long gkey = ((long long)s->device << 8) | key;
  auto it = s->tuned.find(key);
  if (it == s->tuned.end()) {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto jt = g_tuned.find(gkey);
    if (jt != g_tuned.end()) it = s->tuned.insert({key, jt->second}).first;
  }
  if (it != s->tuned.end()) {
    g.variant = it->second.first;
    g.grid_vol = s->sms * it->second.second;
    return ES_DG_OK;
  }
  float best = 1e30f;
  int bv = 0, bm = 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int v = 0; v < nvar; v++) {
    build_tiles(s, g, v);
    g.variant = v;
    int st = upload(s);
    if (st) return st;
    // valid face fluxes for the volume launches being timed
    if (face_launch(s, g)) return ES_DG_ECUDA;
    const int occ = vol_occ(g, v);
    for (int mult = 1; mult <= 2; mult++) {
      g.grid_vol = s->sms * occ * mult;
      if (vol_launch(s, g, 0.0, 0.0)) return ES_DG_ECUDA;  // warm-up
      cudaEventRecord(a, s->stream);
      for (int r = 0; r < 3; r++)
        if (vol_launch(s, g, 0.0, 0.0)) return ES_DG_ECUDA;
      cudaEventRecord(b, s->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) return ES_DG_ECUDA;
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) {
        best = ms;
        bv = v;
        bm = occ * mult;
      }
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  g.variant = bv;
  g.grid_vol = s->sms * bm;
  s->tuned[key] = {bv, bm};
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    g_tuned[gkey] = {bv, bm};
  }
  s->graph_valid = false;
  return ES_DG_OK;
}

// Rebuild descriptors, groups and tables after a membership change.
int rebuild(es_dg_server* s) {
  s->h_members.resize(s->active.size());
  std::vector<int> seen;
  for (size_t m = 0; m < s->active.size(); m++) {
    Member& mb = *s->active[m];
    EsdgLGL L;
    int mixed = 0;
    int st = esdg_member_descriptor(mb.h, mb.dt, &s->h_members[m], &L, &mixed);
    if (st) return st;
    int gi = group_index(s, mb.N, mixed);
    if (gi < 0) {
      Group g;
      g.N = mb.N;
      g.mixed = mixed;
      g.L = L;
      g.grid_face = s->sms * 8;
      s->groups.push_back(g);
      gi = (int)s->groups.size() - 1;
      s->graph_valid = false;
    }
  }
  // groups left without members are dropped (their tuning stays in s->tuned)
  for (size_t gi = 0; gi < s->groups.size();) {
    Group& g = s->groups[gi];
    bool any = false;
    for (auto& m : s->active) any |= (m->N == g.N && m->mixed == g.mixed);
    if (any) {
      gi++;
      continue;
    }
    if (g.d_vt) cudaFree(g.d_vt);
    if (g.d_ft) cudaFree(g.d_ft);
    if (g.d_n) cudaFree(g.d_n);
    s->groups.erase(s->groups.begin() + gi);
    s->graph_valid = false;
  }
  for (Group& g : s->groups) {
    if (g.variant < 0) {
      // first time: tune on the members present (tables are built inside)
      bool any = false;
      for (auto& m : s->active) any |= (m->N == g.N && m->mixed == g.mixed);
      if (any) {
        int st = autotune(s, g);
        if (st) return st;
      } else {
        g.variant = 0;
        g.grid_vol = s->sms;
      }
    }
    build_tiles(s, g, g.variant);
  }
  return upload(s);
}

int launch_step(es_dg_server* s) {
  for (int st = 0; st < 5; st++) {
    for (const Group& g : s->groups)
      if (int r = face_launch(s, g)) return r;
    for (const Group& g : s->groups)
      if (int r = vol_launch(s, g, kA[st], kB[st])) return r;
  }
  return ES_DG_OK;
}

int step(es_dg_server* s) {
  if (!s->use_graph) return launch_step(s);
  if (!s->graph_valid) {
    if (s->graph) {
      cudaGraphExecDestroy(s->graph);
      s->graph = nullptr;
    }
    cudaGraph_t gr;
    cudaError_t e = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(s, e, "begin capture");
    int rc = launch_step(s);
    e = cudaStreamEndCapture(s->stream, &gr);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(s, e, "end capture");
    e = cudaGraphInstantiate(&s->graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return cuda_fail(s, e, "graph instantiate");
    s->graph_valid = true;
  }
  cudaError_t e = cudaGraphLaunch(s->graph, s->stream);
  return e == cudaSuccess ? ES_DG_OK : cuda_fail(s, e, "graph launch");
}

// create and initialise one member (worker thread)
int admit_one(es_dg_server* s, Member& m) {
  const es_dg_request& q = m.req;
  es_dg_mesh mesh{};
  mesh.kx = q.kx;
  mesh.ky = q.ky;
  mesh.kz = q.kz;
  es_dg_physics ph{1.4, 9.81, 287.0, 1.0e5, 0.0, 0.0, 0.0, 1};
  const bool bubble = q.kind != 1;  // kinds 0 and 2: rising bubbles in the 1000 m cube
  if (bubble) {
    for (int d = 0; d < 3; d++) {
      mesh.lo[d] = 0.0;
      mesh.hi[d] = 1000.0;
    }
    mesh.periodic[0] = mesh.periodic[1] = 1;
    mesh.periodic[2] = 0;
    mesh.warp = q.warp;
  } else {  // baroclinic channel stand-in
    mesh.hi[0] = 40000e3;
    mesh.hi[1] = 6000e3;
    mesh.hi[2] = 30e3;
    mesh.periodic[0] = 1;
    ph.f0 = 1e-4;
  }
  // a resident member with the same mesh and order lends its geometry (a device
  // copy instead of the double-double metric computation)
  const es_dg_t* twin = nullptr;
  for (const auto& a : s->active)
    if (a->h && (a->req.kind != 1) == bubble && a->req.kx == q.kx && a->req.ky == q.ky &&
        a->req.kz == q.kz && a->req.N == q.N && (!bubble || a->req.warp == q.warp)) {
      twin = a->h;
      break;
    }
  int st = esdg_create_from(&mesh, q.N, q.precision, &ph, s->stream, twin, &m.h);
  if (st) {
    std::snprintf(s->msg, sizeof(s->msg), "es_dg_create: %s", es_dg_strerror(st));
    return st;
  }
  if (bubble) {
    const double c[3] = {q.centre[0], q.centre[1], q.centre[2]};
    st = es_dg_init_bubble_profile(m.h, q.theta0 > 0 ? q.theta0 : 300.0, q.amp, c,
                                   q.radius > 0 ? q.radius : 250.0,
                                   q.kind == 2 ? ES_DG_BUBBLE_SHARP : ES_DG_BUBBLE_SMOOTH);
  } else {
    st = es_dg_init_channel(m.h);
  }
  if (!st) st = es_dg_cfl_dt(m.h, q.cfl > 0 ? q.cfl : ES_DG_SERVER_DEFAULT_CFL, &m.dt);
  if (st) {
    std::snprintf(s->msg, sizeof(s->msg), "initial state: %s", es_dg_strerror(st));
    es_dg_destroy(m.h);
    m.h = nullptr;
    return st;
  }
  es_dg_info_t info;
  es_dg_get_info(m.h, &info);
  m.N = q.N;
  m.mixed = (q.precision == ES_DG_FP32_MIXED);
  m.ndof = info.ndof;
  return ES_DG_OK;
}

// Tune the group (N, mixed) on a representative member that is created,
// timed and discarded (es_dg_server_warmup).  Worker thread.
int warm_one(es_dg_server* s, int N, int mixed) {
  const long long key = N * 2 + mixed;
  if (s->tuned.count(key)) return ES_DG_OK;
  {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto jt = g_tuned.find(((long long)s->device << 8) | key);
    if (jt != g_tuned.end()) {
      s->tuned[key] = jt->second;
      return ES_DG_OK;
    }
  }
  auto m = std::make_unique<Member>();
  es_dg_request& q = m->req;
  q.kind = 0;
  q.kx = q.ky = q.kz = N <= 4 ? 16 : 8;
  q.N = N;
  q.precision = mixed ? ES_DG_FP32_MIXED : ES_DG_FP64;
  q.cfl = ES_DG_SERVER_DEFAULT_CFL;
  q.amp = 0.5;
  q.centre[0] = q.centre[1] = 500.0;
  q.centre[2] = 350.0;
  q.radius = 250.0;
  q.theta0 = 300.0;
  q.warp = 0.05;
  int st = admit_one(s, *m);
  if (st) return st;
  s->active.push_back(std::move(m));
  st = rebuild(s);  // creates the group and tunes it on this member
  es_dg_destroy(s->active.back()->h);
  s->active.pop_back();
  const int st2 = rebuild(s);  // the tables of the members that stay
  return st ? st : st2;
}

// Read the members' status words (synchronous): a member whose state went
// non-finite (or its density non-positive) is marked to finish with
// ES_DG_ENAN; the others go on.
int poll_flags(es_dg_server* s) {
  s->steps_since_poll = 0;
  const int n = std::min(s->n_table, (int)s->active.size());
  if (n == 0 || !s->d_flags) return ES_DG_OK;
  cudaError_t e = cudaMemcpyAsync(s->h_flags, s->d_flags, sizeof(int) * n, cudaMemcpyDeviceToHost,
                                  s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "status poll");
  for (int m = 0; m < n; m++)
    if (s->h_flags[m] && !s->active[m]->failed) {
      s->active[m]->failed = ES_DG_ENAN;
      std::snprintf(s->msg, sizeof(s->msg), "request %llu: non-finite state after step %d",
                    (unsigned long long)s->active[m]->ticket, s->active[m]->steps_done);
    }
  return ES_DG_OK;
}

void finish(es_dg_server* s, std::unique_ptr<Member>& m, int status) {
  Result res;
  es_dg_result& r = res.r;
  r.status = status;
  r.ticket = m->ticket;
  r.t_submit = m->t_submit - s->t0;
  r.t_admit = m->t_admit - s->t0;
  r.t_finish = now_s() - s->t0;
  r.ndof = m->ndof;
  r.nsteps = m->steps_done;
  r.dt = m->dt;
  if (m->h && status == ES_DG_OK) {
    r.nq = (size_t)m->ndof * 5;
    r.q = (double*)std::malloc(sizeof(double) * r.nq);
    if (!r.q || es_dg_get_state(m->h, r.q, 0) || es_dg_integrals(m->h, r.integrals)) {
      r.status = ES_DG_ECUDA;
    }
  }
  if (m->h) es_dg_destroy(m->h);
  m->h = nullptr;
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= m->bytes;
  s->st.finished++;
  s->st.dof_updates += (double)m->ndof * 5.0 * m->steps_done;
  s->done[m->ticket] = res;
  s->cv.notify_all();
}

void worker(es_dg_server* s) {
  cudaSetDevice(s->device);
  while (true) {
    std::vector<std::unique_ptr<Member>> admit;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait_for(lk, std::chrono::milliseconds(s->active.empty() ? 50 : 0), [&] {
        return s->stop || !s->pending.empty() || !s->active.empty() || !s->warm_jobs.empty();
      });
      if (s->stop && s->pending.empty() && s->active.empty() && s->warm_jobs.empty()) break;
      // warm-up jobs first (the callers wait for them)
      while (!s->warm_jobs.empty()) {
        WarmJob* job = s->warm_jobs.front();
        s->warm_jobs.pop_front();
        lk.unlock();
        int st = ES_DG_OK;
        for (int N : job->orders)
          if (!st) st = warm_one(s, N, job->mixed);
        lk.lock();
        job->status = st;
        job->done = true;
        s->cv.notify_all();
      }
      // FIFO admission by HBM footprint and slots
      while (!s->pending.empty()) {
        Member& head = *s->pending.front();
        if ((int)(s->active.size() + admit.size()) >= s->max_slots) break;
        if (s->used + head.bytes > s->budget) break;
        s->used += head.bytes;
        admit.push_back(std::move(s->pending.front()));
        s->pending.pop_front();
      }
    }
    bool changed = false;
    for (auto& m : admit) {
      m->t_admit = now_s();
      int st = admit_one(s, *m);
      if (st) {
        finish(s, m, st);
        continue;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.admitted++;
      s->active.push_back(std::move(m));
      changed = true;
    }
    // retire cancelled members
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (auto& m : s->active)
        if (s->cancelled.count(m->ticket)) m->req.nsteps = m->steps_done;  // finish now
    }
    // status words: before any member of the table retires, and every 16 steps
    {
      bool due = s->steps_since_poll >= 16;
      for (int m = 0; m < s->n_table && m < (int)s->active.size() && !due; m++)
        due = s->active[m]->steps_done >= s->active[m]->req.nsteps;
      if (due && poll_flags(s) == ES_DG_OK)
        for (auto& m : s->active)
          if (m->failed) m->req.nsteps = m->steps_done;  // finish now, alone
    }
    // retire members that reached their step count
    for (size_t i = 0; i < s->active.size();) {
      if (s->active[i]->steps_done >= s->active[i]->req.nsteps) {
        int status = s->active[i]->failed ? s->active[i]->failed : ES_DG_OK;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          if (s->cancelled.count(s->active[i]->ticket)) status = ES_DG_ECANCELED;
        }
        cudaStreamSynchronize(s->stream);
        finish(s, s->active[i], status);
        s->active.erase(s->active.begin() + i);
        changed = true;
      } else {
        i++;
      }
    }
    if (s->active.empty()) continue;
    if (changed) {
      int st = rebuild(s);
      if (st) {
        s->last_error = st;
        for (auto& m : s->active) finish(s, m, st);
        s->active.clear();
        continue;
      }
    }
    const double ts = now_s();
    int st = step(s);
    if (st) {
      s->last_error = st;
      cudaStreamSynchronize(s->stream);
      for (auto& m : s->active) finish(s, m, st);
      s->active.clear();
      continue;
    }
    for (auto& m : s->active) m->steps_done++;
    s->steps_since_poll++;
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.steps++;
    s->st.launch_seconds += now_s() - ts;
  }
  cudaStreamSynchronize(s->stream);
}

}  // namespace

// ---------------------------------------------------------------------------
extern "C" {

int es_dg_server_create(size_t hbm_budget_bytes, int max_slots, void* cuda_stream,
                        es_dg_server** out) {
  if (!out || max_slots < 1 || hbm_budget_bytes == 0) return ES_DG_EINVAL;
  *out = nullptr;
  es_dg_server* s = new (std::nothrow) es_dg_server();
  if (!s) return ES_DG_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  // the server needs a capturable stream: the legacy default stream is not
  if (cuda_stream) {
    s->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete s;
      return ES_DG_ECUDA;
    }
    s->own_stream = true;
  }
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return ES_DG_ECUDA;
  }
  const char* g = std::getenv("ES_DG_NO_GRAPH");
  s->use_graph = !(g && g[0] == '1');
  const char* v = std::getenv("ES_DG_BATCH_VARIANT");
  if (v && v[0] >= '0' && v[0] <= '9') s->force_variant = v[0] - '0';
  s->t0 = now_s();
  s->worker = std::thread(worker, s);
  *out = s;
  return ES_DG_OK;
}

int es_dg_server_warmup(es_dg_server* s, const int* orders, int n_orders,
                        es_dg_precision precision) {
  if (!s || n_orders < 0 || (n_orders > 0 && !orders)) return ES_DG_EINVAL;
  if (precision != ES_DG_FP64 && precision != ES_DG_FP32_MIXED) return ES_DG_EINVAL;
  WarmJob job;
  for (int i = 0; i < n_orders; i++) {
    if (orders[i] < 1 || orders[i] > 7) return ES_DG_EINVAL;
    job.orders.push_back(orders[i]);
  }
  job.mixed = precision == ES_DG_FP32_MIXED;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->stop) return ES_DG_EINVAL;
  s->warm_jobs.push_back(&job);
  s->cv.notify_all();
  s->cv.wait(lk, [&] { return job.done; });
  return job.status;
}

int es_dg_batch_submit(es_dg_server* s, const es_dg_request* req, uint64_t* ticket) {
  if (!s || !req || !ticket) return ES_DG_EINVAL;
  if (req->N < 1 || req->N > 7 || req->kx < 1 || req->ky < 1 || req->kz < 1 || req->nsteps < 0 ||
      req->kind < 0 || req->kind > 2 ||
      (req->precision != ES_DG_FP64 && req->precision != ES_DG_FP32_MIXED))
    return ES_DG_EINVAL;
  auto m = std::make_unique<Member>();
  m->req = *req;
  m->bytes = estimate_bytes(*req);
  m->t_submit = now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (m->bytes > s->budget) return ES_DG_ENOMEM;  // could never be admitted
  if ((int)s->pending.size() >= 1 << 20) return ES_DG_EBUSY;
  m->ticket = s->next_ticket++;
  *ticket = m->ticket;
  s->st.submitted++;
  s->pending.push_back(std::move(m));
  s->cv.notify_all();
  return ES_DG_OK;
}

int es_dg_batch_poll(es_dg_server* s, uint64_t ticket, es_dg_result* out) {
  if (!s || !out) return ES_DG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) return ticket > 0 && ticket < s->next_ticket ? ES_DG_PENDING : ES_DG_EINVAL;
  *out = it->second.r;
  s->done.erase(it);
  return ES_DG_OK;
}

int es_dg_batch_wait(es_dg_server* s, uint64_t ticket, double timeout_s, es_dg_result* out) {
  if (!s || !out) return ES_DG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double>(timeout_s));
  while (true) {
    auto it = s->done.find(ticket);
    if (it != s->done.end()) {
      *out = it->second.r;
      s->done.erase(it);
      return ES_DG_OK;
    }
    if (ticket == 0 || ticket >= s->next_ticket) return ES_DG_EINVAL;
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return ES_DG_ETIMEOUT;
  }
}

int es_dg_batch_cancel(es_dg_server* s, uint64_t ticket) {
  if (!s) return ES_DG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto it = s->pending.begin(); it != s->pending.end(); ++it)
    if ((*it)->ticket == ticket) {
      Result res;
      res.r.status = ES_DG_ECANCELED;
      res.r.ticket = ticket;
      s->done[ticket] = res;
      s->pending.erase(it);
      s->cv.notify_all();
      return ES_DG_OK;
    }
  s->cancelled[ticket] = 1;
  return ES_DG_OK;
}

void es_dg_result_free(es_dg_result* r) {
  if (!r) return;
  std::free(r->q);
  r->q = nullptr;
  r->nq = 0;
}

int es_dg_server_stats(es_dg_server* s, es_dg_server_stats_t* out) {
  if (!s || !out) return ES_DG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->active = (int)s->active.size();
  out->pending = (int)s->pending.size();
  out->bytes_in_use = s->used;
  out->last_error = s->last_error;
  std::memcpy(out->error, s->msg, sizeof(out->error));
  return ES_DG_OK;
}

void es_dg_server_destroy(es_dg_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // requests still waiting are cancelled; running ones finish their steps
    while (!s->pending.empty()) {
      Result res;
      res.r.status = ES_DG_ECANCELED;
      res.r.ticket = s->pending.front()->ticket;
      s->done[res.r.ticket] = res;
      s->pending.pop_front();
    }
    s->cv.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& kv : s->done) std::free(kv.second.r.q);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  for (Group& g : s->groups) {
    if (g.d_vt) cudaFree(g.d_vt);
    if (g.d_ft) cudaFree(g.d_ft);
    if (g.d_n) cudaFree(g.d_n);
  }
  if (s->d_members) cudaFree(s->d_members);
  if (s->d_flags) cudaFree(s->d_flags);
  if (s->h_flags) cudaFreeHost(s->h_flags);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
