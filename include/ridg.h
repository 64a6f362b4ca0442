/*
 * ridg.h -- C ABI of the GB300 nodal discontinuous-Galerkin RTM library.
 *
 * The library solves the first-order acoustic pressure-velocity system
 *     dp/dt + rho c^2 div v = f(t) delta(x - x0),      rho dv/dt + grad p = 0
 * (Sec. 2, Eqs. waveSyst1-2) on unstructured tetrahedra with the nodal DG scheme of
 * Sec. 3.1 (Eqs. dgLocalSchemeP/U), the multi-rate Adams-Bashforth local time stepping of
 * Sec. 3.2 (Eqs. updateAB, updateABcoarse, Algorithm 1), and accumulates the classical
 * (Eq. imageP) and characteristic (Eqs. imageQ, charact) imaging conditions of one RTM shot
 * with the AB3-exact increments of Sec. 3.3 (Eq. updateABcorr).  Every step of the time loop
 * runs in CUDA kernels for sm_103a; the host only prepares the mesh and schedules launches.
 *
 * Conventions
 *  - Every function returns an int status: RIDG_OK (0) or a negative RIDG_E_* code.  The
 *    message of the last failure of the calling thread is returned by ridg_last_error().
 *    No C++ exception crosses this interface.
 *  - Arrays are C-contiguous.  "host" pointers are read or written by the CPU; "device"
 *    pointers must be CUDA device memory of the current device.  The library copies every
 *    input it keeps; the caller keeps ownership of all buffers it passes.
 *  - Element fields are laid out [K][4][Np] with the fields (p, vx, vy, vz) and the nodes in
 *    the reference order: equidistant lattice order (t slowest, then s, r fastest) of the
 *    warp-and-blend nodes of Sec. 3.1.  Np = (N+1)(N+2)(N+3)/6.
 *  - Local face f of tetrahedron (v0,v1,v2,v3) is spanned by the vertices
 *    f=0:(v0,v1,v2), f=1:(v0,v1,v3), f=2:(v1,v2,v3), f=3:(v0,v2,v3).
 *  - Handles are not thread safe; use one solver per host thread and stream.
 */
#ifndef RIDG_H
#define RIDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define RIDG_OK 0
#define RIDG_E_INVALID_ARG -1 /* a size, pointer or option is out of range */
#define RIDG_E_BAD_MESH -2    /* degenerate/inverted element, non-manifold face, boundary code on an interior face */
#define RIDG_E_OOM -3         /* device or host memory could not be allocated */
#define RIDG_E_CUDA -4        /* a CUDA call failed (message holds cudaGetErrorString) */
#define RIDG_E_UNSTABLE -5    /* a non-finite value or energy growth was detected */
#define RIDG_E_TIMEOUT -6     /* a bounded wait gave up (ridg_server_wait's timeout) */
#define RIDG_E_NOT_FOUND -7   /* a source or receiver lies outside the mesh */
#define RIDG_E_BUSY -8        /* a shot server's queue is full */
#define RIDG_E_INTERNAL -9    /* a consistency check of the solver's tables failed (RIDG_DEBUG=1) */

/* boundary-condition codes per local face (Sec. 2): 0 = automatic (interior where a neighbour
 * exists, else the default code), 1 = free surface p = 0, 2 = transparent p - rho c n.v = 0
 * (Eq. ABC), 3 = rigid wall n.v = 0. */
#define RIDG_BC_AUTO 0
#define RIDG_BC_FREE 1
#define RIDG_BC_TRANSPARENT 2
#define RIDG_BC_RIGID 3

/* working precision of the fields and kernels */
#define RIDG_F32 0
#define RIDG_F64 1

typedef struct ridg_mesh ridg_mesh;
typedef struct ridg_solver ridg_solver;

/* Returns the message of the last failing call of this thread ("" if none). */
const char* ridg_last_error(void);

/* Library version string. */
const char* ridg_version(void);

/* ------------------------------------------------------------------ mesh (host only)
 * Creates a tetrahedral mesh (Sec. 3.1: Omega = union of the cells D_k).
 *   xyz      host double [n_vert][3]  vertex coordinates
 *   tet      host int64  [K][4]       vertex indices; every element must have positive
 *                                      orientation det[v1-v0, v2-v0, v3-v0] > 0
 *   face_bc  host int8   [K][4] or NULL  boundary code per local face (RIDG_BC_*); a non-zero
 *                                      code on a face shared by two elements is RIDG_E_BAD_MESH
 *   default_bc                          code of unmatched faces whose face_bc is 0
 * Faces are matched by their vertex triples.  Errors: RIDG_E_INVALID_ARG, RIDG_E_BAD_MESH. */
int ridg_mesh_create(const double* xyz, int64_t n_vert, const int64_t* tet, int64_t K, const int8_t* face_bc,
                     int8_t default_bc, ridg_mesh** out);
void ridg_mesh_destroy(ridg_mesh* mesh);
/* Number of boundary faces, interior faces of the mesh (host only). */
int ridg_mesh_counts(const ridg_mesh* mesh, int64_t* n_boundary_faces, int64_t* n_interior_faces);

/* Point location (host only): for each of the n points xyz[3*i..3*i+2] the element that contains
 * it (barycentric coordinates >= -1e-12; the lowest element index when the point lies on a face,
 * edge or vertex shared by several) in elem_out[i], or -1 outside the mesh, and its reference
 * coordinates (r, s, t) on the reference tetrahedron with vertices (-1,-1,-1), (1,-1,-1), (-1,1,-1),
 * (-1,-1,1) in rst_out[3*i..] (may be NULL).  Sources and receivers are placed with this rule
 * (Eq. sourceTerm, receiver interpolation).  A uniform grid index is built on the first call and
 * kept with the mesh.  Errors: RIDG_E_INVALID_ARG. */
int ridg_mesh_locate(ridg_mesh* mesh, const double* xyz, int64_t n, int64_t* elem_out, double* rst_out);

/* ------------------------------------------------------------------ reference element (host only)
 * Operators of the reference tetrahedron of order N (Sec. 3.1 and the appendix), computed by the
 * library's own setup code.  Any output pointer may be NULL.
 *   rst   [Np][3]   node coordinates          D     [3][Np][Np]  D_r, D_s, D_t
 *   M     [Np][Np]  mass matrix               LIFT  [Np][4*Nfp]  M^{-1} E (face masses on a
 *   fmask [4][Nfp]  face node indices                            2-D reference triangle of area 2) */
int ridg_reference_operators(int N, double* rst, double* D, double* M, double* LIFT, int32_t* fmask);

/* ------------------------------------------------------------------ solver */
typedef struct ridg_options {
  int32_t dtype;        /* RIDG_F32 (default) or RIDG_F64 */
  double cfl;           /* C in Delta t_k = C l_k / ((N+1)^2 c_k) (Sec. 5.1); <= 0 selects 0.15 */
  int32_t n_levels_max; /* maximum number of multi-rate levels (Sec. 3.2); <= 0 selects 3 */
  int32_t image_mask;   /* images a shot accumulates: RIDG_IMAGE_P | RIDG_IMAGE_Q; 0 selects both */
  double tau_scale;     /* multiplies the penalty parameters tau_p = 1/Zbar, tau_v = Zbar of the
                           upwind fluxes (Sec. 3.1, Eqs. weakFormP/V); <= 0 selects 1 (upwind) */
  int32_t contraction;  /* RIDG_F32 only: RIDG_CONTRACT_TENSOR (0, default) runs the D_r/D_s/D_t and
                           LIFT products on tensor cores with FP32 accumulation: the three-term TF32
                           split up to N = 4, the FP16 split below from N = 5 (faster there and more
                           accurate); RIDG_CONTRACT_TENSOR_TF32 the TF32 split at every order;
                           RIDG_CONTRACT_CUDA_CORES runs them as plain FP32 FMAs;
                           RIDG_CONTRACT_TENSOR_BF16 on tensor cores as a BF16 hi + lo split (three
                           m16n8k16 products, FP32 accumulation: about 2^-16 relative per product);
                           RIDG_CONTRACT_TENSOR_FP16 as an FP16 hi + lo split (about 2^-22), each
                           element column of each operand tile scaled by a power of two into FP16's
                           range before the split and the scale removed from the FP32 sums */
  int32_t reserved[3];
} ridg_options;
#define RIDG_CONTRACT_TENSOR 0
#define RIDG_CONTRACT_CUDA_CORES 1
#define RIDG_CONTRACT_TENSOR_BF16 2
#define RIDG_CONTRACT_TENSOR_FP16 3
#define RIDG_CONTRACT_TENSOR_TF32 4

#define RIDG_IMAGE_P 1 /* classical image, Eq. imageP */
#define RIDG_IMAGE_Q 2 /* characteristic image, Eq. imageQ */

typedef struct ridg_info {
  int32_t N, Np, Nfp, n_levels;
  int64_t K;
  double dt_local, dt_global;  /* Delta t_local and Delta t_global = 2^(n_levels-1) Delta t_local */
  int64_t level_count[8];      /* elements per level, level 1 (coarsest) first */
  int64_t n_boundary_faces;
  int64_t device_bytes;        /* device memory held by the solver (fields, history, traces, tables) */
  int64_t n_half_step;         /* elements with a finer neighbour (they also write half-step traces) */
} ridg_info;

/* Creates a solver for order N (1..6) with piecewise-constant c, rho per element (host double
 * [K] each, positive).  Sets up the reference operators, geometric factors (inverse Jacobian,
 * normals, J_f/J), face connectivity, multi-rate levels (coarsest level each element's bound
 * allows, then moved finer until neighbours differ by at most one level) and uploads them.
 * cuda_stream: a cudaStream_t cast to uintptr_t (0 = default stream); every kernel of this
 * solver runs on it.  The state starts at rest at t = 0.
 * Errors: RIDG_E_INVALID_ARG, RIDG_E_BAD_MESH, RIDG_E_OOM, RIDG_E_CUDA. */
int ridg_solver_create(const ridg_mesh* mesh, int N, const double* c, const double* rho, const ridg_options* opt,
                       uintptr_t cuda_stream, ridg_solver** out);
void ridg_solver_destroy(ridg_solver* s);
int ridg_solver_info(const ridg_solver* s, ridg_info* info);
/* Level (1 = coarsest) of every element, host int32 [K]. */
int ridg_solver_levels(const ridg_solver* s, int32_t* levels);
/* Physical node coordinates, host double [K][Np][3]. */
int ridg_solver_nodes(const ridg_solver* s, double* xyz);

/* ------------------------------------------------------------------ state access
 * ridg_set_state: q host double [K][4][Np]; sets the fields, recomputes the traces, resets the
 *   time to t = 0 and the right-hand-side history to zero.
 * ridg_set_history: host double [K][4][Np] each (may be NULL = zero): the right-hand sides one
 *   and two level steps before the current time (each element at its own level's step), the
 *   values Eq. updateAB needs before the first step.
 * ridg_eval_rhs: host double in [K][4][Np] -> out [K][4][Np]: the right-hand side of Eqs.
 *   dgLocalSchemeP/U (forward tau, no source) of the given fields, evaluated by the CUDA kernel.
 *   Does not change the solver's state.
 * ridg_step: advances n_global global steps (Algorithm 1; one fused kernel launch per step of the
 *   finest level), asynchronously on the solver's stream.
 * ridg_get_state: copies the fields to host double [K][4][Np] (synchronises the stream).
 * ridg_set_state_device / ridg_get_state_device: the same with a device double [K][4][Np] buffer
 *   owned by the caller (for instance a torch tensor's data_ptr()); asynchronous on the solver's
 *   stream (ridg_set_state_device keeps no reference to q_dev once the stream has passed it). */
int ridg_set_state(ridg_solver* s, const double* q);
int ridg_set_state_device(ridg_solver* s, const double* q_dev);
int ridg_get_state_device(ridg_solver* s, double* q_dev);
int ridg_set_history(ridg_solver* s, const double* rhs_prev1, const double* rhs_prev2);
int ridg_eval_rhs(ridg_solver* s, const double* q, double* rhs_out);
int ridg_step(ridg_solver* s, int64_t n_global);
int ridg_get_state(ridg_solver* s, double* q_out);
/* Discrete energy sum_k J_k/2 (p^T M p/(rho c^2) + rho v^T M v), accumulated in FP64 on the device. */
int ridg_energy(ridg_solver* s, double* energy);

/* The same energy of the solver's current fields, for callers that cannot allocate device memory
 * when they need it: a host application that gives the library a fixed device-memory budget and
 * owns every allocation, or a time-critical stepping loop in which cudaMalloc/cudaFree must not run
 * (they can block the host and synchronise the device).  The paper has no counterpart: this is an
 * interface variant of ridg_energy.
 *   energy_dev  device double[1] owned by the caller; written asynchronously on the solver's stream.
 * Allocates no device memory: its scratch (per-block partial sums) is a fixed 32 KiB device array
 * that every GPU loading the library keeps until exit.  Solvers with more than 1,048,576 element
 * slots (elements padded to multiples of 32 per level) are rejected with RIDG_E_INVALID_ARG.  The
 * first call on a device looks up the scratch array's device address with that device current;
 * make that first call before any stream capture.  Calls share the scratch array: calls that overlap
 * on the GPU (other streams or unordered solvers on the same device) race.
 * Errors: RIDG_E_INVALID_ARG, RIDG_E_CUDA. */
int ridg_energy_noalloc(ridg_solver* s, double* energy_dev);

/* ------------------------------------------------------------------ one RTM shot (Sec. 2, Sec. 4.3)
 * Source at xyz (Eq. waveSyst1, L2-projected Dirac of Eq. sourceTerm) with wavelet f(t):
 *   kind RIDG_SRC_RICKER (0): f(t) = amplitude (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
 *     tau = t - t_peak;
 *   kind RIDG_SRC_SAMPLED (1): f(t) = amplitude * interpolant of samples[n] at t = n sample_dt
 *     (n = 0 .. n_samples-1; 4-point Lagrange interpolation in time, zero outside the samples);
 *     samples is a host array, copied by the call.
 * Receivers: rec_xyz host double [nrec][3]; traces are sampled at t_n = n Delta t_global for
 * n = 0 .. n_t-1 with n_t = ridg_trace_len(s, t_final) = ceil(t_final / Delta t_global) + 1.
 *
 * ridg_rtm_shot runs (i) the forward source run with receiver sampling and the recording of the
 * traces (p, n.v) on every boundary face at every evaluation time of its element, two global steps
 * past t_final; (ii) the backward source run from the saved final state, whose boundary faces take
 * the recorded traces as their exterior state; (iii) the backward receiver run that re-injects the
 * observed traces (cubic Lagrange interpolation in time); (ii) and (iii) run in lockstep in one
 * fused kernel per step, which also accumulates the two images over [t_image_start, t_final].
 *   observed   host double [nrec][n_t] or NULL (= re-inject the modelled traces)
 *   traces_out host double [nrec][n_t] or NULL
 *   image_p    host double [K][Np] or NULL: classical image int p_S p_R dt (Eq. imageP)
 *   image_q    host double [K][Np] or NULL: characteristic image int q^-_S q^+_R dt (Eq. imageQ),
 *              q^{+/-} = p +/- c rho (e_up . v)
 *              (an image left out of the solver's image_mask is not accumulated and reads zero)
 *   e_up       host double [3] or NULL (= (0,0,-1): z is depth)
 * The images are accumulated in FP64.  The call synchronises the stream before returning.
 * Errors: RIDG_E_INVALID_ARG, RIDG_E_NOT_FOUND, RIDG_E_OOM (boundary-trace arena), RIDG_E_CUDA,
 * RIDG_E_UNSTABLE. */
#define RIDG_SRC_RICKER 0
#define RIDG_SRC_SAMPLED 1
typedef struct ridg_source {
  double xyz[3];
  double f0, t_peak, amplitude; /* f0, t_peak: RIDG_SRC_RICKER only */
  int32_t kind;                 /* RIDG_SRC_RICKER (0) or RIDG_SRC_SAMPLED */
  int32_t reserved;
  double sample_dt;             /* RIDG_SRC_SAMPLED: sample spacing (> 0) */
  int64_t n_samples;            /* RIDG_SRC_SAMPLED: number of samples (>= 1) */
  const double* samples;        /* RIDG_SRC_SAMPLED: host double [n_samples] */
} ridg_source;

/* Forward modelling: the forward source run of ridg_rtm_shot alone (no boundary records, no
 * backward runs), from rest at t = 0 to t_final, with the receiver pressures sampled at
 * t_n = n Delta t_global.  traces_out: host double [nrec][n_t], n_t = ridg_trace_len(s, t_final).
 * Leaves the solver's fields at t_final.  Errors: RIDG_E_INVALID_ARG, RIDG_E_NOT_FOUND, RIDG_E_CUDA. */
int ridg_forward(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                 double* traces_out);

int64_t ridg_trace_len(const ridg_solver* s, double t_final);
int ridg_rtm_shot(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                  double t_image_start, const double* observed, double* traces_out, double* image_p,
                  double* image_q, const double* e_up);
/* Same shot with device buffers: observed, traces_out (double [nrec][n_t]) and image_p, image_q
 * (double [K][Np]) are device pointers (observed/traces_out/images may be NULL).  Nothing is
 * copied between host and device except the small per-shot tables; the call returns after the
 * work is enqueued (synchronise the solver's stream before reading the outputs). */
int ridg_rtm_shot_device(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec,
                         double t_final, double t_image_start, const double* observed_dev, double* traces_dev,
                         double* image_p_dev, double* image_q_dev, const double* e_up);

/* ------------------------------------------------------------------ several shots in lockstep
 * n_shots (1 .. RIDG_MAX_BATCH) shots of this solver's model, each as ridg_rtm_shot (its own source,
 * wavelet, receivers, observed traces and outputs; Sec. 2 per shot), over one record length t_final,
 * one image window [t_image_start, t_final] and one e_up.  The shots advance in lockstep: every fine
 * step is a single launch of the fused step kernel over the active elements of all of them (FP32
 * tensor-core contractions; with FP64 or CUDA-core FP32 the shots are stepped one after the other
 * within each fine step), so the finest-level steps, which cover few elements, fill more of the GPU
 * and the element tables are read once per step.  Every shot's results are those of the same shot
 * run alone by ridg_rtm_shot, bit for bit.  The solver keeps device state for each shot of its
 * largest batch (fields, histories, traces, boundary records, images) until it is destroyed (a shot
 * server gives it back from idle slots when it needs the memory).  ridg_last_shot_stats then counts
 * the whole batch.  A solver with a trace budget (ridg_set_trace_budget) runs batches of one shot
 * only.  The paper runs one shot at a time.
 *   shots[i].observed, .traces_out, .image_p, .image_q: as the arguments of ridg_rtm_shot (host
 *   buffers) or of ridg_rtm_shot_device (device buffers, for ridg_rtm_shots_device); rec_xyz is a
 *   host array either way.
 * Errors: as ridg_rtm_shot; RIDG_E_INVALID_ARG for n_shots outside 1 .. RIDG_MAX_BATCH. */
#define RIDG_MAX_BATCH 4
typedef struct ridg_shot_io {
  ridg_source source;
  const double* rec_xyz; /* [nrec][3] host */
  int64_t nrec;
  const double* observed; /* [nrec][n_t] or NULL (re-inject the modelled traces) */
  double* traces_out;     /* [nrec][n_t] or NULL */
  double* image_p;        /* [K][Np] or NULL */
  double* image_q;        /* [K][Np] or NULL */
} ridg_shot_io;
int ridg_rtm_shots(ridg_solver* s, int32_t n_shots, const ridg_shot_io* shots, double t_final,
                   double t_image_start, const double* e_up);
/* Device-buffer form: returns after the work is enqueued on the solver's stream. */
int ridg_rtm_shots_device(ridg_solver* s, int32_t n_shots, const ridg_shot_io* shots, double t_final,
                          double t_image_start, const double* e_up);

/* Counters of the last shot: DOF updates (elements updated x 4 x Np, both wavefields counted in
 * the backward phase), fused-kernel launches and total kernel launches. */
typedef struct ridg_shot_stats {
  int64_t dof_updates_forward, dof_updates_backward;
  int64_t fused_launches, kernel_launches;
  int64_t n_global, boundary_trace_bytes;
  /* with profiling on: CUDA-event time (ms) and count of the sampled fused launches that cover
   * every element (all levels active), forward (one wavefield) and backward (two wavefields) */
  double prof_forward_ms, prof_backward_ms;
  int64_t prof_forward_launches, prof_backward_launches;
  /* boundary-trace records beyond the device budget (ridg_set_trace_budget): the chunks they were
   * moved in (1: all on the device) and the bytes copied to host memory (the backward run copies
   * the ones it reads back) */
  int64_t trace_chunks, host_trace_bytes;
  /* 1 when the shot's time stepping ran as one CUDA-graph launch (ridg_set_graph_replay) */
  int64_t graph_replay;
} ridg_shot_stats;
/* Synchronises the solver's stream, then returns the counters of the last shot. */
int ridg_last_shot_stats(const ridg_solver* s, ridg_shot_stats* stats);

/* CUDA-graph replay of the time stepping of repeated shots (on != 0; off by default).  A shot or
 * lockstep batch (ridg_rtm_shot_device, ridg_rtm_shots_device, and the shots of a server's slots,
 * whose buffers stay in place) whose launches would take exactly the arguments of the previous one
 * -- the same number of shots, record length, image window, e_up and image mask, per shot the same
 * wavelet, receiver count and device buffers (observed, traces, images) -- captures its stream work
 * (every kernel launch, memset and device copy from the start of the forward run to the images)
 * into a CUDA graph the second time, and launches that graph the times after: one launch instead of
 * one per fine step.  Source and receiver positions and the observed data may differ, since the
 * kernels read them from device tables uploaded before the stepping.  The results are those of the
 * launches it replaces, bit for bit.  Profiling (ridg_set_profiling), a trace budget, the parts of
 * a group and solvers on the default stream (which cannot be captured) run without graphs.  The paper has no counterpart.  Errors: RIDG_E_INVALID_ARG,
 * RIDG_E_CUDA (the capture or instantiation failed). */
int ridg_set_graph_replay(ridg_solver* s, int32_t on);

/* Device memory for the boundary-trace records of a shot (Sec. 4.3; the forward run records the
 * traces of every boundary face of every active element at every fine step, the backward source run
 * replays them).  device_bytes = 0 (the default) keeps every record on the device.  With
 * device_bytes > 0 and a shot whose records need more, the records of consecutive fine steps are
 * grouped into chunks of at most device_bytes / 2: during the forward run each full chunk except the
 * last two is copied to pinned host memory (allocated by the solver, the size of all records, kept
 * for later shots) on a second stream while the next chunk fills the other half of the device
 * buffer, and the backward run copies them back, one chunk ahead, in reverse order.  Results are
 * bit for bit those of the shot with every record on the device.  A shot fails with
 * RIDG_E_INVALID_ARG when device_bytes / 2 cannot hold the records of one fine step, and with
 * RIDG_E_OOM when the host memory cannot be allocated.  device_bytes < 0: RIDG_E_INVALID_ARG.
 * Admission by device memory (ridg_server_*) counts at most device_bytes for the records. */
int ridg_set_trace_budget(ridg_solver* s, int64_t device_bytes);

/* Profiling: when every > 0, every every-th global step the fused launch that covers all elements
 * is bracketed by CUDA events on the solver's stream; 0 turns it off (default). */
int ridg_set_profiling(ridg_solver* s, int32_t every);

/* ------------------------------------------------------------------ velocity gradient
 * The paper migrates with the imaging condition; these calls give the gradient of a least-squares
 * trace misfit with respect to the per-element velocity, as the exact discrete adjoint of the
 * library's scheme (Sec. 3.1 right-hand side, Sec. 3.2 AB3; with several rate levels Algorithm 1
 * with its half-step traces).  The velocity enters through rho c^2 in the pressure equation; the
 * time step, the levels and the penalty parameters tau_p, tau_v (and the impedance of I_Q) keep the
 * values of the model the solver was created with. */

/* Velocity per element (host double [K], > 0) in rho c^2; see above for what stays frozen.
 * Invalidates the last misfit forward run.  Because the time step and the levels stay those of the
 * creation model, an element's Courant number on its level's step, Dt_l (N+1)^2 c_k / l_k (l_k its
 * smallest height), may not exceed 4/3 of the solver's CFL constant (0.2 at the default 0.15; AB3
 * with this step rule was measured stable up to 0.22 and unstable at 0.25): a faster element is
 * rejected with RIDG_E_INVALID_ARG, naming it, instead of silently running an unstable scheme. */
int ridg_set_velocity(ridg_solver* s, const double* c);
/* out = A^T lam, the transposed right-hand-side operator (no source), host double [K][4][Np] each
 * in the reference node numbering.  The parity check of the adjoint kernels. */
int ridg_eval_adjoint_rhs(ridg_solver* s, const double* lam, double* out);
/* Forward run from rest with the source, receiver traces y_r^n at every step t_n = n Dt
 * (n = 0 .. n_t-1, n_t from ridg_trace_len) and the misfit
 *   J = 1/2 Dt sum_n sum_r (y_r^n - observed_r^n)^2      (observed: host double [nrec][n_t], nrec >= 1).
 * Keeps n_checkpoints (<= 0 selects 16) snapshots of the state for ridg_misfit_backward.
 * traces_out (host double [nrec][n_t]) may be NULL.  Any number of rate levels (Algorithm 1; the
 * global step is Dt).  Errors: RIDG_E_INVALID_ARG (missing receivers or data), RIDG_E_NOT_FOUND,
 * RIDG_E_UNSTABLE. */
int ridg_misfit_forward(ridg_solver* s, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                        const double* observed, int32_t n_checkpoints, double* misfit, double* traces_out);
/* grad (host double [K]) = dJ/dc of the last ridg_misfit_forward: the adjoint recursion
 *   lambda^m = lambda^{m+1} + Dt A^T sum_s a_s lambda^{m+1+s} - Dt sum_r (y_r^m - d_r^m) l(x_r),
 * run backward from m = n_t-1, recomputing the forward states segment by segment from the
 * checkpoints, with dJ/dc_k = -(2/c_k) sum_n lambda^{n+1}_p,k . (A (q^{n+1} - q^n source-free))_p,k.
 * With several rate levels the same gradient comes from reverse accumulation over the fine steps of
 * Algorithm 1 (the transposed trace pushes, updates and right-hand sides of each fine step; the
 * levels, the time step and tau stay frozen); each segment's right-hand sides are kept on the device
 * (segment length x NL field arrays).
 * Leaves the solver's fields at the first checkpoint's segment (set the state again before stepping).
 * May be called again for the same forward run.  RIDG_E_INVALID_ARG without a valid forward run
 * (none yet, or the velocity changed since). */
int ridg_misfit_backward(ridg_solver* s, double* grad);

/* ------------------------------------------------------------------ shot server
 * The paper's unit of work is the RTM shot (Sec. 2; a survey migrates many shots into one image).
 * A server serves shot requests on a set of slots.  A slot is a solver: one model (mesh, c, rho,
 * order, precision) with its own CUDA stream and device buffers (fields, histories, traces, the
 * boundary-trace arena of Sec. 4.3), kept resident between shots.  Slots are numbered by model:
 * several solvers built from the same inputs serve one model concurrently.  Each slot has a worker
 * thread; an idle slot takes the oldest waiting request of its model, so requests that arrive
 * while others run start as soon as a slot of their model is free, and the shots of different
 * slots overlap on the device (their solvers must use different non-default streams for that).
 * Admission by device memory: before a shot starts, the memory it still needs (the arena grows
 * with the record length) must be free; if it is not, the buffers of idle slots are released and,
 * while other slots run, the request waits for them to finish; if the memory cannot be found it
 * completes with RIDG_E_OOM.  While a request waits for memory, idle slots start no new requests.
 * A shot's results do not depend on the slot or on the other shots.  The server has no
 * counterpart in the paper.  While a server exists, its solvers must not be used by any other
 * call.  One thread should submit and wait per server (the calls are thread-safe, but the last
 * error message is per thread). */
typedef struct ridg_server ridg_server;

typedef struct ridg_shot_request {
  ridg_source source;
  const double* rec_xyz; /* [nrec][3] host; copied at submission */
  int64_t nrec;
  double t_final, t_image_start;
  const double* observed; /* [nrec][n_t] host or NULL (the modelled traces); copied at submission */
  double* traces_out;     /* [nrec][n_t] host or NULL; owned by the caller, written before completion */
  double* image_p;        /* [K][Np] host or NULL (K, Np of the request's model); as traces_out */
  double* image_q;        /* [K][Np] host or NULL; as traces_out */
  const double* e_up;     /* [3] or NULL for (0, 0, -1); copied at submission */
  int32_t model;          /* model number of the slots that may serve the request (0 for one model) */
  int32_t reserved;
} ridg_shot_request;

typedef struct ridg_request_timing {
  double queued_s; /* submission to start */
  double run_s;    /* start to completion (admission, the shot and the copies into the host buffers) */
  double total_s;  /* submission to completion */
  double start_s;  /* start, in seconds since the server was created */
  double end_s;    /* completion, in seconds since the server was created */
  int64_t slot;    /* the slot that served the request */
} ridg_request_timing;

/* Creates a server with one slot (solver s, model 0) and its worker thread; at most max_queued
 * requests may wait (>= 1). */
int ridg_server_create(ridg_solver* s, int64_t max_queued, ridg_server** out);
/* Creates a server over n_slots solvers; models[i] (>= 0) is the model number of solvers[i]
 * (NULL: all model 0).  Solvers of one model must have the same element count, order, levels and
 * time step (checked) and should be built from the same mesh, media and options.  Each solver
 * appears once. */
int ridg_server_create_slots(ridg_solver* const* solvers, const int32_t* models, int64_t n_slots, int64_t max_queued,
                             ridg_server** out);
/* Queues a request and returns its ticket.  RIDG_E_BUSY when max_queued requests are waiting;
 * RIDG_E_INVALID_ARG for a malformed request or a model no slot serves (checked again, with the
 * solver, when it runs). */
int ridg_server_submit(ridg_server* sv, const ridg_shot_request* req, int64_t* ticket);
/* A slot that takes a request also takes up to max_batch - 1 later waiting requests of its model
 * with the same t_final, t_image_start and e_up, and runs them together as one lockstep batch
 * (ridg_rtm_shots: one merged launch per fine step); each request's results are those it gets
 * alone.  max_batch in 1 .. RIDG_MAX_BATCH; 1 (the default) runs one shot at a time.  Admission
 * counts the memory of the whole batch; a batch that fails (a request the library rejects, or too
 * little memory for all of them) runs its requests one by one, each completing with its own status.
 * Errors: RIDG_E_INVALID_ARG. */
int ridg_server_set_batch(ridg_server* sv, int32_t max_batch);
/* Waits at most timeout_s seconds (< 0: without limit) for a request.  When it has completed,
 * releases the ticket, fills timing (may be NULL) and returns the request's own status (0, or the
 * error it ran into, with its message in ridg_last_error); RIDG_E_TIMEOUT if it has not completed
 * in time (the ticket stays valid); RIDG_E_INVALID_ARG for an unknown ticket. */
int ridg_server_wait(ridg_server* sv, int64_t ticket, double timeout_s, ridg_request_timing* timing);
/* Finishes the running requests, drops the queued ones (their buffers are not written) and frees
 * the server; the solvers can be used again afterwards. */
int ridg_server_destroy(ridg_server* sv);

/* ------------------------------------------------------------------ domain decomposition (Sec. 4.2)
 * One shot on a mesh split into parts, each part advanced by its own solver (on its own device, or
 * several parts on one device), as the paper runs one part per device of a cluster.  After every
 * fine step the traces (p, n.v) that a part's elements pushed across faces to elements of another
 * part are copied into that part's face inboxes; only the elements advanced at that step have
 * pushed, and with the lumping below the steps that advance the finest level only copy nothing.
 * Both backward wavefields use the same partition, so the images need no transfer (Sec. 4.2).  The
 * union of the parts' traces and images is the shot of one solver over the whole mesh. */
#define RIDG_MAX_PARTS 64
typedef struct ridg_group ridg_group;

/* part_out (host int32 [K]): the part of each element, for n_parts parts (1..RIDG_MAX_PARTS).
 * Weights 2^(l-1) per element of level l (l = 1 coarsest: its right-hand-side evaluations per
 * global step), levels as ridg_solver_create assigns them (opt: cfl, n_levels_max; NULL for the
 * defaults) for order N and velocity c (host double [K]); every finest element, or connected group
 * of them, is lumped with its face neighbours and kept in one part unless the lump outweighs half a
 * part's share; the lumps are split by weighted recursive coordinate bisection of their weighted
 * vertex centroids (across the longest extent, at the weighted median; the paper uses METIS with
 * the same weights and lumping).  Host only.  Errors: RIDG_E_INVALID_ARG. */
int ridg_partition(const ridg_mesh* mesh, int N, const double* c, const ridg_options* opt, int32_t n_parts,
                   int32_t* part_out);

typedef struct ridg_group_info {
  int32_t n_parts;
  int32_t reserved;
  int64_t elements[RIDG_MAX_PARTS];        /* elements each part advances */
  int64_t ghosts[RIDG_MAX_PARTS];          /* elements of other parts next to them */
  int64_t interface_faces[RIDG_MAX_PARTS]; /* faces across which each part pushes to another part */
  /* the last shot: */
  int64_t dof_updates;     /* all parts, both phases */
  int64_t transfer_steps;  /* fine steps (of all wavefield runs) after which traces were copied */
  int64_t silent_steps;    /* fine steps that needed no copy (finest level only, lumping held) */
  int64_t transfer_bytes;  /* bytes copied between parts */
} ridg_group_info;

/* A group of n_parts solvers for the parts part[K] (host int32, values 0..n_parts-1, each part
 * non-empty) of mesh, with the media, order and options of ridg_solver_create; part i lives on CUDA
 * device devices[i] (host int32 [n_parts]; NULL: all on the current device) with a stream of its
 * own.  Parts on different devices copy traces between devices (peer copies).  The levels and time
 * step are those of the whole mesh.  Errors: RIDG_E_INVALID_ARG, RIDG_E_BAD_MESH, RIDG_E_OOM,
 * RIDG_E_CUDA. */
int ridg_group_create(const ridg_mesh* mesh, int N, const double* c, const double* rho, const ridg_options* opt,
                      const int32_t* part, int32_t n_parts, const int32_t* devices, ridg_group** out);
/* One RTM shot over the whole mesh with the arguments and host buffers of ridg_rtm_shot (traces_out
 * [nrec][n_t], image_p / image_q [K][Np], any of them NULL).  One host thread per part drives it;
 * the call returns when every part has finished.  A source or receiver belongs to the part of the
 * element that contains it.  Errors as ridg_rtm_shot. */
int ridg_group_rtm_shot(ridg_group* g, const ridg_source* src, const double* rec_xyz, int64_t nrec, double t_final,
                        double t_image_start, const double* observed, double* traces_out, double* image_p,
                        double* image_q, const double* e_up);
int ridg_group_info_get(const ridg_group* g, ridg_group_info* out);
/* n_t of a record of t_final seconds (as ridg_trace_len); Np through np_out (may be NULL). */
int64_t ridg_group_trace_len(const ridg_group* g, double t_final, int32_t* np_out);
void ridg_group_destroy(ridg_group* g);

/* ------------------------------------------------------------------ failure injection (tests)
 * A host-side failure point that fires once, through the same error path as the failure it stands
 * for, after `after` passes (0: the next one); nothing touches the GPU.  Points: "alloc" (a device
 * allocation: RIDG_E_OOM), "arena" (the boundary-trace arena of a shot: RIDG_E_OOM), "admission" (the
 * shot server's memory admission refuses a request: RIDG_E_OOM), "exchange" (a part group's interface
 * transfer: RIDG_E_CUDA from ridg_group_rtm_shot, every other part released), "none" (disarm).  The
 * environment variable RIDG_FAULT=<point>[:<after>] arms one when the library loads.  The calls
 * after a fired failure work as before.  No counterpart in the paper.  Errors: RIDG_E_INVALID_ARG. */
int ridg_inject_fault(const char* point, int64_t after);
/* The armed point (0 none, 1 alloc, 2 arena, 3 admission, 4 exchange). */
int ridg_fault_armed(void);

#ifdef __cplusplus
}
#endif
#endif /* RIDG_H */
