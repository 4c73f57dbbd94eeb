/*
 * es_dg.h -- C ABI of the GB300 entropy-stable DG Euler + buoyancy library.
 *
 * The library evaluates the semi-discrete right-hand side of the entropy-stable
 * discontinuous Galerkin method (Section 3, Eq. (nm:semi)) on structured boxes
 * of curvilinear hexahedra with (N+1)^3 LGL nodes, and advances it with the
 * Carpenter-Kennedy five-stage fourth-order low-storage Runge-Kutta scheme.
 * All arithmetic runs in CUDA kernels on one GPU; the host only launches.
 *
 * Conventions
 *   - Every function returns int: ES_DG_OK (0), a negative error code, or (for
 *     es_dg_batch_poll only) ES_DG_PENDING (> 0).  es_dg_strerror() names it.
 *   - State layout q[e][v][n] in double: v = 0..4 is rho, rho u, rho v, rho w, E
 *     (E includes rho g z, Section 2); n = i + Nq (j + Nq k) with Nq = N + 1;
 *     e = ex + Kx (ey + Ky ez).  Element ex spans
 *     [lo_x + ex (hi_x - lo_x)/Kx, lo_x + (ex+1)(hi_x - lo_x)/Kx] before warping.
 *   - The caller owns every pointer it passes; the library copies in and out.
 *     "on_device" = 1 means the pointer is device memory of the handle's GPU,
 *     0 means host memory (pageable or pinned).
 *   - A handle is not thread-safe; calls on one handle are ordered on its stream
 *     and return before the GPU work finishes unless stated otherwise.
 *   - Precision changes only internal arithmetic; the interface is always double.
 */
#ifndef ES_DG_H
#define ES_DG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ES_DG_OK = 0,
  ES_DG_PENDING = 1,     /* es_dg_batch_poll: request not finished yet */
  ES_DG_EINVAL = -1,     /* bad argument */
  ES_DG_ENOMEM = -2,     /* device allocation failed or over budget */
  ES_DG_ECUDA = -3,      /* a CUDA call failed */
  ES_DG_ENAN = -4,       /* non-finite or non-physical state detected */
  ES_DG_ETIMEOUT = -5,   /* a bounded device wait ran out */
  ES_DG_EBUSY = -6,      /* server queue full */
  ES_DG_ECANCELED = -7   /* request cancelled */
};

typedef enum {
  ES_DG_FP64 = 0,        /* all arithmetic in FP64 */
  ES_DG_FP32_MIXED = 1   /* flux pairs and derivative sums in FP32; state,
                            RK accumulation, pressure and energy recovery in FP64 */
} es_dg_precision;

/* Structured box of Kx x Ky x Kz hexahedra.  periodic[d] = 1 joins the two d
 * faces, 0 makes them reflecting walls.  warp > 0 displaces every node by
 *   x += warp Lx sin(2 pi y'/Ly) sin(2 pi z'/Lz), y += warp Ly sin(2 pi z'/Lz) sin(2 pi x'/Lx),
 *   z += warp Lz sin(2 pi x'/Lx) sin(2 pi y'/Ly)   (primes: offsets from lo, all
 * evaluated at the unwarped point). */
typedef struct {
  int kx, ky, kz;
  double lo[3], hi[3];
  int periodic[3];
  double warp;
} es_dg_mesh;

/* Gas, gravity and rotation constants (Section 2).  gamma = cp/cv, g the
 * gravitational acceleration (phi = g z), R the gas constant, p0 the reference
 * pressure of the initial states, Coriolis parameter f = f0 + beta (y - y0)
 * about z.  dissipation = 1 adds matrix dissipation to the interface flux
 * (Section 3), 0 keeps it entropy-conservative.  NULL selects gamma = 1.4,
 * g = 9.81, R = 287, p0 = 1e5, f0 = beta = y0 = 0, dissipation = 1. */
typedef struct {
  double gamma, g, R, p0, f0, beta, y0;
  int dissipation;
} es_dg_physics;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes` or NULL; free releases it.  NULL
 * allocator = cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, void* ctx);
  void* ctx;
} es_dg_allocator;

typedef struct es_dg es_dg_t;

typedef struct {
  int N, Nq, np;           /* order, nodes per direction, nodes per element */
  int nelem;               /* elements */
  long long ndof;          /* nodes = nelem * np (the paper counts DOF this way) */
  long long nfaces;        /* interior, periodic and wall faces */
  size_t device_bytes;     /* device memory held by the handle */
  int precision;
} es_dg_info_t;

/* Create a solver on the current CUDA device.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream).  Builds node coordinates, curl-form
 * metric terms (Kopriva), face normals and the LGL operators on the device.
 * N in 1..7; at most 2^30 elements (so face indices fit in 32 bits) and a
 * warp amplitude in [0, 0.15), else ES_DG_EINVAL.  On error *out is NULL. */
int es_dg_create(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                 const es_dg_physics* physics, const es_dg_allocator* allocator,
                 void* cuda_stream, es_dg_t** out);
void es_dg_destroy(es_dg_t* h);
int es_dg_get_info(const es_dg_t* h, es_dg_info_t* info);

/* Copy the state in or out (layout above, nelem*5*np doubles). */
int es_dg_set_state(es_dg_t* h, const double* q, int on_device);
int es_dg_get_state(es_dg_t* h, double* q, int on_device);

/* Rising-bubble initial state on the device (Section 5.1, Eq. (smooth-rb-ic)):
 * isentropic background theta0, cosine theta perturbation of amplitude amp
 * (K) and radius `radius` about `centre`; pressure unperturbed; u = 0. */
int es_dg_init_bubble(es_dg_t* h, double theta0, double amp, const double centre[3],
                      double radius);
/* The same with the profile chosen: ES_DG_BUBBLE_SMOOTH is es_dg_init_bubble;
 * ES_DG_BUBBLE_SHARP is the step of Section 5.1, Eq. (sharp-rb-ic): theta0 + amp
 * for r <= radius, theta0 outside (a discontinuity the entropy-stable flux must
 * carry without a limiter).  Any other profile: ES_DG_EINVAL. */
enum { ES_DG_BUBBLE_SMOOTH = 0, ES_DG_BUBBLE_SHARP = 1 };
int es_dg_init_bubble_profile(es_dg_t* h, double theta0, double amp, const double centre[3],
                              double radius, int profile);
/* Synthetic baroclinic-channel state (Section 5.2 configuration; the benchmark's
 * own balanced-jet formulas are not in the paper, so this is a stand-in):
 * isothermal columns p = p0 exp(-z/H(y)), H(y) = 7500 m + 60 m (1 - tanh((y -
 * 3000 km)/600 km)), rho = p/(g H), zonal wind in geostrophic balance
 * u = -g z H'(y)/(f H) with f = f0 + beta (y - y0), plus the perturbation
 * 1 m/s exp(-((x - 2000 km)^2 + (y - 2500 km)^2)/(600 km)^2); v = w = 0.
 * Needs f != 0 somewhere (ES_DG_EINVAL when f0 = beta = 0).  A mixed handle gets
 * the channel state at rest as its background (es_dg_set_background). */
int es_dg_init_channel(es_dg_t* h);
/* The channel state with the perturbation's amplitude amp (m/s; 1 in
 * es_dg_init_channel, 0 the balanced jet alone) and the mixed path's background
 * chosen: ES_DG_BACKGROUND_REST as es_dg_init_channel, ES_DG_BACKGROUND_JET the
 * balanced jet itself, carried with its flow (es_dg_set_moving_background; whole
 * meshes only, ES_DG_EINVAL on a partition).  No background in FP64 mode.
 * ES_DG_EINVAL: amp not finite, another background value, f0 = beta = 0. */
enum { ES_DG_BACKGROUND_REST = 0, ES_DG_BACKGROUND_JET = 1 };
int es_dg_init_channel_ex(es_dg_t* h, double amp, int background);

/* Hydrostatic background of the mixed-precision path (the perturbation-variable
 * formulation the paper suggests for 32-bit runs, Section 5.2).  From q_bg the
 * library keeps rho_bg and b_bg = rho/(2p) and evaluates, once and in FP64, the
 * right-hand side of the same state at rest, (rho_bg, 0, p_bg/(gamma-1) + rho_bg phi).
 * Every later mixed-precision evaluation computes rhs(q) = rhs(q_bg at rest) +
 * [rhs(q) - rhs(q_bg at rest)], the bracket in FP32 with the pressure and gravity
 * differences formed exactly in perturbation variables, so FP32 rounding is
 * relative to the perturbation.  In exact arithmetic the result is unchanged.
 * es_dg_init_bubble sets the unperturbed atmosphere and es_dg_init_channel the
 * channel state at rest as background automatically.  No effect in FP64 mode.
 * Synchronous when on_device = 0.  es_dg_clear_background returns to plain FP32. */
int es_dg_set_background(es_dg_t* h, const double* q_bg, int on_device);
/* A moving background: q_bg itself, flow included (Section 5.2's perturbation
 * formulation extended to a background that carries a flow, e.g. the channel's
 * balanced jet, whose density and energy right-hand sides cancel convective
 * fluxes far larger than themselves).  The library evaluates rhs(q_bg) once in
 * FP64 (every component, the Coriolis force of its momentum included) and forms
 * every flux of the FP32 bracket rhs(q) - rhs(q_bg) as an exact difference in
 * perturbation variables (rho', m', E', u', p', b'), so FP32 rounding is relative
 * to q - q_bg.  Requirements of the formulation: q_bg continuous across faces and
 * tangential at walls (u_bg . n = 0 there), as a state given per node of one
 * mesh is when it comes from a smooth field of position with that property.
 * Whole meshes only (ES_DG_EINVAL on a partition; the server's batched kernels
 * carry only a background at rest).  No effect in FP64 mode.  Synchronous when
 * on_device = 0; q_bg (nelem*5*np doubles) is copied. */
int es_dg_set_moving_background(es_dg_t* h, const double* q_bg, int on_device);
int es_dg_clear_background(es_dg_t* h);

/* One evaluation of the right-hand side dq/dt of Eq. (nm:semi) at state q
 * (not the handle's state), written to rhs.  Both pointers host or both device
 * per on_device.  Synchronous when on_device = 0. */
int es_dg_rhs(es_dg_t* h, const double* q, double* rhs, int on_device);

/* Time step of the handle's state from the contravariant signal speeds,
 *   dt = C (xi_1 - xi_0) / max over nodes and directions d of
 *        (|u . Ja^d| + c |Ja^d|) / J,
 * which on an affine element of edge h is C h (xi_1 - xi_0) / (2 (|u_d| + c)).
 * Synchronous.  -ES_DG_ENAN if the state has a non-positive pressure. */
int es_dg_cfl_dt(es_dg_t* h, double C, double* dt);

/* Advance the handle's state by nsteps LSRK(5,4) steps of size dt (Section 3).
 * Asynchronous on the handle's stream; each stage is one interface-flux launch
 * and one volume launch with the RK update fused in. */
int es_dg_step(es_dg_t* h, double dt, int nsteps);

/* Wait for the handle's stream.  Returns ES_DG_ETIMEOUT if, since the last
 * call, a bounded device wait of the pipelined volume kernels ran out (their
 * tile copies never completed; the kernel stopped and the state is not
 * valid), ES_DG_ENAN if a stage update of this handle (es_dg_step) produced a
 * state value that is an infinity or a NaN, or a density that is not positive
 * (the kernels keep stepping; the state is not valid), ES_DG_ECUDA on a CUDA
 * error, else ES_DG_OK.  The timeout flag is process-wide per device, the
 * state flag is the handle's; the call clears both. */
int es_dg_sync(es_dg_t* h);

/* Test hook for the failure path above: the next single-mesh volume launch
 * (any handle, this process) registers 16 bytes more on its first tile
 * barrier than its copies deliver, so every CTA's bounded wait runs out
 * (about a second), the kernel stops without touching memory further, and
 * the next es_dg_sync returns ES_DG_ETIMEOUT.  The state of that handle is
 * then undefined; the context stays usable.  One-shot. */
void es_dg_debug_inject_wait_timeout(void);

/* Test hook for the numeric helpers that the kernels use in place of FP64-pipe
 * instructions: out[i] = helper(in[i]) for i < n, on device arrays (in: doubles,
 * or floats for F2D and F2D_POS; out: floats for D2F and D2F_TAIL, else
 * doubles), asynchronous on cuda_stream.  k is the power of two for LDEXP.
 *   D2F       double -> float, round to nearest even, for |x| < 2^128 (a
 *             rounding past FLT_MAX gives +-inf; results below the float normal
 *             range flush to +-0; larger magnitudes, infinities and NaNs are
 *             outside the helper's domain and give an unspecified value)
 *   F2D       float -> double (exact; zero and subnormal floats give +-0)
 *   LDEXP     x 2^k (exact for normal x and results; +-inf / NaN kept;
 *             subnormal inputs and results flush to +-0; overflow to +-inf)
 *   RCP       1/x to about one rounding (MUFU seed + cubic refinement)
 *   RCP_LO    1/x to about 2^-39 (one Newton step)
 *   D2F_TAIL  0 <= u < 2^128 to float by mantissa truncation (0 below the float
 *             normal range)
 *   F2D_POS   positive normal float -> double (exact)
 * ES_DG_EINVAL for an unknown helper, n < 0 or missing arrays. */
enum { ES_DG_NUM_D2F = 0, ES_DG_NUM_F2D = 1, ES_DG_NUM_LDEXP = 2, ES_DG_NUM_RCP = 3,
       ES_DG_NUM_RCP_LO = 4, ES_DG_NUM_D2F_TAIL = 5, ES_DG_NUM_F2D_POS = 6 };
int es_dg_debug_numeric(int which, const void* in, void* out, long long n, int k,
                        void* cuda_stream);

/* Global integrals of the handle's state: mass, total energy, entropy
 * (sum over elements of the quadrature of rho, E and -rho s/(gamma-1)).
 * Synchronous. */
int es_dg_integrals(es_dg_t* h, double out[3]);

/* Device geometry for inspection: x[e][3][n], J[e][n], Ja[e][d][c][n] (double).
 * Any pointer may be NULL.  Synchronous when on_device = 0. */
int es_dg_geometry(es_dg_t* h, double* x, double* J, double* Ja, int on_device);

/* Launch a single kernel of the right-hand side on the handle's state: which =
 * 0 interface flux (every face), 1 volume (writes the rhs buffer), 2 volume with
 * the fused RK update at stage `stage` (0..4) and step dt; on a partition also
 * 3 the interface flux of every face whose outside state needs no trace, and 4
 * that of the faces of its remote planes (3 then 4 equals 0: a caller can run 3
 * while the traces are in flight, Section 4.3's overlap of the exchange with
 * the work that does not depend on it).  ES_DG_EINVAL for another value. */
int es_dg_launch(es_dg_t* h, int which, int stage, double dt);

/* ---- Domain decomposition (Section 4.3: elements split among processes, face
 * traces exchanged every stage).  A mesh is cut into slabs of whole x element
 * layers; each slab is a handle of its own whose cut x planes are "remote":
 * their outside state is a trace, 5 x (N+1)^2 values per face of the plane,
 * received from the neighbouring slab before every stage.  Node positions,
 * metric terms, face geometry and arithmetic are those of the whole mesh, so
 * partitioned stepping reproduces the whole-mesh result bit for bit.  Traces
 * live in caller-owned device buffers, which lets the caller move them with
 * device copies (es_dg_partitions_*: all slabs on one GPU and one stream) or
 * with any transport between processes (pack, send / receive, then es_dg_launch
 * for the stage).  A periodic x wraps from the last slab to the first. */

/* Handle of x element layers [x_begin, x_end) of `mesh` (0 <= x_begin < x_end <=
 * kx).  Its low plane is remote if x_begin > 0 or x is periodic, its high plane
 * if x_end < kx or x is periodic (a slab holding every layer is a whole mesh).
 * Other arguments as es_dg_create.  es_dg_step on a handle with a remote plane
 * returns ES_DG_EINVAL; es_dg_rhs and es_dg_launch use the received traces as
 * they stand and return ES_DG_EINVAL until es_dg_set_traces gave them. */
int es_dg_create_partition(const es_dg_mesh* mesh, int N, es_dg_precision precision,
                           const es_dg_physics* physics, int x_begin, int x_end,
                           const es_dg_allocator* allocator, void* cuda_stream, es_dg_t** out);
/* The slab's layer range, remote flags (low, high) and the length in doubles of
 * one plane's trace: ky * kz * nv * (N+1)^2, laid out [face a + ky b][slot][face
 * node i_y + (N+1) i_z]; slots 0-4 the conserved state, and for FP32-mixed
 * handles (nv = 7) slots 5-6 the background rho_bg and p_bg of the node, which a
 * mixed slab needs for the faces of its cut planes (its background's own
 * right-hand side is evaluated at the first stage after they arrived).  Any
 * output pointer may be NULL. */
int es_dg_partition_info(const es_dg_t* h, int* x_begin, int* x_end, int remote[2],
                         long long* trace_len);
/* Register the trace buffers (device, trace_len doubles each, 8-byte aligned,
 * owned by the caller and alive while the handle uses them).  send_* are written
 * by es_dg_pack_traces, recv_* are read by the interface kernel; the pair of a
 * plane that is not remote may be NULL.  ES_DG_EINVAL if a remote plane lacks one. */
int es_dg_set_traces(es_dg_t* h, double* send_lo, double* send_hi, double* recv_lo,
                     double* recv_hi);
/* Stream-ordered: ES_DG_TRACE_STATE writes the state of the slab's first layer
 * at its low face nodes into send_lo and of its last layer at its high face nodes
 * into send_hi (remote planes only).  ES_DG_TRACE_GEOMETRY writes the high plane's
 * face geometry (normals, scalings, geopotential: the same length) into send_hi;
 * the neighbour hands it to es_dg_accept_geometry_trace, once, before stepping. */
enum { ES_DG_TRACE_STATE = 0, ES_DG_TRACE_GEOMETRY = 1 };
int es_dg_pack_traces(es_dg_t* h, int what);
/* Take recv_lo as the low plane's face geometry (the whole mesh evaluates a face
 * from the element below it, here the neighbour's).  No-op without a remote low
 * plane. */
int es_dg_accept_geometry_trace(es_dg_t* h);
/* All slabs of one mesh on one GPU: parts[0..P-1] in x order, created on one
 * stream, traces set.  connect exchanges the face geometry (once, synchronous);
 * exchange packs every state trace and copies each into its neighbour's receive
 * buffer (device-to-device, stream-ordered); step advances all slabs by nsteps
 * LSRK steps with an exchange before every stage.  ES_DG_EINVAL if the slabs do
 * not cover the mesh in order or a trace buffer is missing. */
int es_dg_partitions_connect(es_dg_t* const* parts, int P);
int es_dg_partitions_exchange(es_dg_t* const* parts, int P);
int es_dg_partitions_step(es_dg_t* const* parts, int P, double dt, int nsteps);

const char* es_dg_strerror(int status);

/* ---- batched ensembles and the continuous-batching server -------------------
 * A server keeps many solves resident on the device and advances all of them
 * together: per LSRK stage, one persistent interface launch and one persistent
 * volume launch per (polynomial order, precision) group walk device work
 * tables of (member, tile) entries; one LSRK step is captured once as a CUDA
 * graph and replayed, and admitting or retiring a solve rewrites the tables,
 * not the graph.  Tile shapes (elements per CTA) and grid sizes are chosen per
 * group by an autotuner that times launches on the resident solves.  Requests
 * are admitted first come, first served when their estimated device footprint
 * fits under the budget and a slot is free; requests arriving while others run
 * join the batch at the next step (continuous batching).  Results carry the
 * final state and the submit / admit / finish times.  Each member's arithmetic
 * is independent of the others, so a result is the same alone and in a mix. */
typedef struct es_dg_server es_dg_server;

/* Courant number of requests that give none.  With the es_dg_cfl_dt rule,
 * C = 0.5 lies on the stability boundary of LSRK(5,4) on unwarped isotropic
 * meshes for N >= 4 (a 1e-10 perturbation grows by 1e5 to overflow within 300
 * steps at N = 4..7), C = 0.45 and below are stable for every order; requests
 * of mixed orders default to 0.4. */
#define ES_DG_SERVER_DEFAULT_CFL 0.4

typedef struct {
  int kind;                  /* 0 = rising bubble (1000 m cube, periodic x/y, walls z),
                                1 = baroclinic channel stand-in (40000 x 6000 x 30 km,
                                    periodic x, walls y/z, f0 = 1e-4),
                                2 = sharp rising bubble (as 0, Eq. (sharp-rb-ic)) */
  int kx, ky, kz, N;         /* elements per direction, order (1..7) */
  es_dg_precision precision;
  int nsteps;                /* LSRK steps to run */
  double cfl;                /* Courant number for dt (0 = ES_DG_SERVER_DEFAULT_CFL); dt
                                fixed at admission */
  double amp, centre[3], radius, theta0;  /* bubble: amplitude (K), centre, radius, theta0 */
  double warp;               /* bubble mesh warp (fraction of the edge) */
} es_dg_request;

typedef struct {
  int status;                /* ES_DG_OK, or the error that ended the request */
  uint64_t ticket;
  double t_submit, t_admit, t_finish;  /* seconds since server creation */
  long long ndof;            /* nodes of the mesh */
  int nsteps;                /* steps completed */
  double dt;
  double integrals[3];       /* mass, energy, entropy of the final state */
  double* q;                 /* final state (host, layout of es_dg_get_state); free with
                                es_dg_result_free */
  size_t nq;
} es_dg_result;

typedef struct {
  long long submitted, admitted, finished, steps;
  int active, pending;
  double dof_updates;        /* sum over finished requests of ndof * 5 * steps */
  double launch_seconds;     /* host time spent launching steps */
  size_t bytes_in_use;       /* estimated footprint of admitted requests */
  int last_error;
  char error[96];            /* text of the last failure, if any */
} es_dg_server_stats_t;

/* Start a server on the current device with a device-memory budget and a
 * maximum number of resident solves.  It runs on cuda_stream, which must be a
 * created stream (graph capture), or, with NULL, on a non-blocking stream of
 * its own. */
int es_dg_server_create(size_t hbm_budget_bytes, int max_slots, void* cuda_stream,
                        es_dg_server** out);
/* Tune the batched kernels of the given polynomial orders (each 1..7) and
 * precision before requests arrive, so that the first request of each order
 * does not wait for the autotuner: for every order not tuned yet, a
 * representative rising-bubble member (16^3 elements at N <= 4, 8^3 above) is
 * created, the tile shape and grid size are timed on it, and it is discarded.
 * Blocks until done.  The choice is kept for the process (every server on
 * this device uses it). */
int es_dg_server_warmup(es_dg_server* s, const int* orders, int n_orders,
                        es_dg_precision precision);
/* Queue a request (copied); -ES_DG_ENOMEM if it can never fit the budget,
 * -ES_DG_EBUSY if the queue is full.  Thread-safe. */
int es_dg_batch_submit(es_dg_server* s, const es_dg_request* req, uint64_t* ticket);
/* ES_DG_PENDING (> 0) until the request is done; then ES_DG_OK and *out owns
 * the result (release its state with es_dg_result_free).  Thread-safe. */
int es_dg_batch_poll(es_dg_server* s, uint64_t ticket, es_dg_result* out);
/* Blocking poll with a timeout (seconds); -ES_DG_ETIMEOUT when it runs out. */
int es_dg_batch_wait(es_dg_server* s, uint64_t ticket, double timeout_s, es_dg_result* out);
/* A request whose state turns non-finite (or whose density turns non-positive)
 * during a step is finished early with status -ES_DG_ENAN, without a state;
 * the server reads the members' status words before a member retires and every
 * 16 steps, and the other members go on unaffected. */
/* Cancel a queued or running request (its result gets -ES_DG_ECANCELED). */
int es_dg_batch_cancel(es_dg_server* s, uint64_t ticket);
void es_dg_result_free(es_dg_result* r);
int es_dg_server_stats(es_dg_server* s, es_dg_server_stats_t* out);
/* Cancel queued requests, finish running ones, stop the scheduler and free. */
void es_dg_server_destroy(es_dg_server* s);

/* ---- allocation-free entry point -------------------------------------------
 * The paper has no counterpart to this function; it exists for callers that
 * cannot allocate device memory (a memory pool they do not own, a framework
 * that forbids cudaMalloc on its hot path, an exhausted allocator).
 *
 * es_dg_integrals_noalloc computes the same three integrals as es_dg_integrals
 * (mass, total energy, entropy) from caller-owned device arrays, without a
 * handle and without allocating: q[e][v][n] (state), J[e][n] and x[e][3][n]
 * (as returned by es_dg_geometry with on_device = 1), for the mesh, order and
 * physics given (physics NULL = defaults).  out3 is caller-owned device memory
 * for 3 doubles, written asynchronously on cuda_stream (a cudaStream_t, NULL =
 * legacy default stream); synchronise the stream before reading it.
 *
 * Scratch: the per-element partial sums live in a static device array sized
 * for ES_DG_NOALLOC_MAX_ELEMS elements (3 doubles each, 6 MiB), present on
 * every GPU that loads the library until the process exits.  Meshes with more
 * elements, and physics that es_dg_create would reject (gamma <= 1, R <= 0,
 * p0 <= 0), get -ES_DG_EINVAL before any CUDA call.  Each call made while
 * cuda_stream is not capturing looks up the array's device address
 * (cudaGetSymbolAddress) with the current device, so a device reset, which may
 * move the array, is picked up; a call made during a capture reuses the
 * address of the last call outside one, so make the first call on each device
 * before any stream capture, and again after a device reset.  All calls share
 * the one array: calls whose work overlaps on the GPU (different streams
 * without ordering) race and must be serialised by the caller. */
#define ES_DG_NOALLOC_MAX_ELEMS 262144
int es_dg_integrals_noalloc(const es_dg_mesh* mesh, int N, const es_dg_physics* physics,
                            const double* q, const double* J, const double* x, double* out3,
                            void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
