/*
 * libapiccontact — the APIC augury contact step of Tupek, Koester & Mosby,
 * "A momentum preserving frictional contact algorithm based on affine
 * particle-in-cell grid transfers" (arXiv 2108.02259), on NVIDIA GB300.
 *
 * One call maps the predicted generalized velocity V = {v_p, C_p} of the
 * contact particles (finite-element boundary nodes, Sec. 2 intro) to the
 * preferred velocity
 *
 *     V_hat = V + G V + sum_{n=1..N} G W_n,        G = H - I        (Sec. 2.3)
 *
 * where H is one APIC particle-to-grid / grid-to-particle transfer pair on a
 * quadratic B-spline background grid of spacing h (Sec. 2.1.2, App. B) and
 * W_{m+1} is the undesirable part of V_hat_m - V under the Coulomb-friction
 * cone (Sec. 2.4).  The caller forms the augury acceleration
 * (V_hat - V) / tau itself (Sec. 2.2, eq. apic_accel).
 *
 * C_p is the APIC affine matrix B_p D_p^{-1}; with the quadratic B-splines
 * D_p = (h^2/2) I (App. B), so B_p = (h^2/2) C_p.  C is row-major 3x3:
 * C[9p + 3a + b] = d v_a / d x_b.
 *
 * Conventions for every entry point:
 *   - No exceptions cross the ABI.  Every call returns an apic_status;
 *     on failure apic_last_error() holds a message for the calling thread.
 *   - The caller owns every pointer it passes.  The library keeps none past
 *     the call.  Scratch (grid, sort buffers) is owned by the context and
 *     grows on demand (cudaMalloc, or the caller's allocator given to
 *     apic_set_allocator); it counts against the context's HBM budget.
 *   - Array pointers are device pointers on the context's device unless the
 *     APIC_HOST_PTRS flag is set.  Work is queued on the caller's CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream).
 *   - A context is not thread-safe; use one per thread.
 */
#ifndef APICCONTACT_H
#define APICCONTACT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t apic_status;
#define APIC_OK 0
#define APIC_ERR_INVALID_ARG (-1)   /* bad size, pointer, flag or value   */
#define APIC_ERR_OUT_OF_MEMORY (-2) /* device allocation or budget failed */
#define APIC_ERR_CUDA (-3)          /* a CUDA runtime call failed         */
#define APIC_ERR_TIMEOUT (-4)       /* a bounded wait gave up             */
#define APIC_ERR_ADMISSION (-5)     /* the HBM budget cannot hold it now  */
#define APIC_ERR_NOT_READY (-6)     /* a request has not completed yet    */

/* Flags of apic_step_args.flags */
#define APIC_FP64 (1u << 0)          /* v, C, m, nrm (in and out) are double; all arithmetic FP64.
                                        Without it they are float and the transfers run in FP32
                                        (positions as int cell + FP32 offset, FP64 node momentum
                                        at nodes two or more bodies touch).                        */
#define APIC_HOST_PTRS (1u << 1)     /* every array pointer is host memory: the call copies in,
                                        computes, copies out and synchronises the stream.          */
#define APIC_VARIANT_PIC (1u << 2)   /* PIC transfers (Sec. 2.1.1): no affine term, C unchanged.   */
#define APIC_VARIANT_SEP23 (1u << 3) /* Sec. 2.3 separation rule instead of the Sec. 2.4 cone:
                                        W = Delta if Delta_v . n > 0, else 0.                      */
#define APIC_DETERMINISTIC (1u << 5) /* Bitwise-reproducible results (FP32 path only; not in the
                                        paper): node sums are added as 64-bit fixed-point integers,
                                        exactly and in any order, with a power-of-two scale per
                                        scene and pass; the transfer kernel runs its first variant
                                        (no autotuning).  A scene's outputs then depend only on its
                                        own inputs: the same bits alone, in any batch, with graphs
                                        or dependent launch on or off, from run to run on one GPU
                                        model.  Costs one host synchronisation at the end of the
                                        step.  A scene whose terms grow past the scale's headroom
                                        within one pass is repeated with a wider one; if that also
                                        fails (or inputs are non-finite) the call returns
                                        APIC_ERR_INVALID_ARG and leaves the outputs of every scene
                                        in the call untouched.  Statistics (apic_stats) are still
                                        FP64 sums.                                                 */
#define APIC_CHECK (1u << 6)         /* Also validate v, C and nrm: every component finite, each
                                        normal 0 or of unit length (|n|^2 within 1e-3 of 1);
                                        otherwise APIC_ERR_INVALID_ARG.  Positions, masses and body
                                        ids are always validated.  Reads v, C and nrm once more.   */

#define APIC_PARTITIONED (1u << 8)  /* apic_contact_step_batched only: the scenes are partitions of
                                        the particles of ONE scene (any split; a spatial one keeps
                                        the shared part of the grid small), all with the same h,
                                        n_bodies, mu and mu_pair table.  Each partition keeps its
                                        own sparse grid; after every particle-to-grid transfer
                                        (eq. massToGrid with the momenta, and each P2G of the Sec.
                                        2.3 series) the nodes of grid blocks active in several
                                        partitions are summed across them (the halo exchange a
                                        spatial decomposition over devices needs once per
                                        transfer pair), so every partition sees the whole scene's
                                        grid and the outputs equal those of one call on the whole
                                        scene, up to FP32 summation order.  Statistics are per
                                        partition.  Not with APIC_DETERMINISTIC.                    */
#define APIC_MASS_NORMALS (1u << 7) /* nrm may be NULL (and is not read): the normals come from
                                        each body's grid mass instead (not in the paper, whose
                                        normals come from the FE surface, Sec. 2.3): after the mass
                                        P2G, n_p = -g/|g| with g the gradient of body b's grid mass
                                        (eq. massToGrid over that body) interpolated at x_p, where
                                        |g| h > 0.5 rho_p (rho_p that mass interpolated at x_p), and
                                        0 inside the body.  About the outermost particle layer of a
                                        body sampled at node spacing h/2.  apic_mass_normals gives
                                        the same normals (any threshold) in the caller's order.    */

typedef struct apic_ctx apic_ctx;

/* One contact step of one scene.
 *   n         number of particles (>= 0; 0 is a no-op).
 *   n_bodies  1..32; body[p] in [0, n_bodies).  Bodies only matter for the
 *             multi-body node bookkeeping and the per-pair friction table.
 *   n_iter    N >= 0 augury iterations: N + 1 transfer pairs (Sec. 2.3).
 *   body      [n] int32.
 *   x         [n*3] double positions, xyz interleaved.  Grid nodes sit at
 *             h * (i, j, k) for all integers (unbounded grid, App. B).
 *   v, C      [n*3], [n*9] predicted velocity and affine matrix (float, or
 *             double with APIC_FP64).
 *   m         [n] masses, > 0.
 *   nrm       [n*3] outward unit normals of surface nodes, 0 for interior
 *             nodes (Sec. 2.3); may be NULL with APIC_MASS_NORMALS.
 *   v_out, C_out  [n*3], [n*9] results; may alias v, C.
 *   h         grid spacing > 0.   mu  scalar friction coefficient >= 0.
 *   mu_pair   NULL, or HOST pointer to n_bodies*n_bodies doubles (symmetric):
 *             per-body-pair friction, blended per particle by the mass of the
 *             other bodies its stencil sees (the paper has one scalar mu).
 *   flags     APIC_* above.
 */
typedef struct {
  int64_t n;
  int32_t n_bodies;
  int32_t n_iter;
  const int32_t* body;
  const double* x;
  const void* v;
  const void* C;
  const void* m;
  const void* nrm;
  void* v_out;
  void* C_out;
  double h;
  double mu;
  const double* mu_pair;
  uint32_t flags;
} apic_step_args;

/* Diagnostics of one step (FP64 reductions on the device).
 *   P = sum m v;  L = sum m [ x cross v + (h^2/2) axial(C) ],
 *   axial(C) = (C_zy - C_yz, C_xz - C_zx, C_yx - C_xy)  — the angular
 *   momentum the grid sees (Sec. 2.1.2).  Requesting stats synchronises. */
typedef struct {
  double P_in[3], P_out[3], L_in[3], L_out[3];
  int64_t multibody_nodes; /* grid nodes with mass from two or more bodies */
  int64_t active_blocks;   /* 4x4x4-node grid blocks allocated this step   */
  int64_t work_items;      /* (grid block, body) particle segments         */
  double E_in, E_out;      /* generalised kinetic energy (1/2) sum m (|v|^2 + (h^2/2) |C|_F^2),
                              FP64, of the inputs and of the outputs          */
} apic_stats;

/* Per-context kernel timing (CUDA events on the caller's stream), for the
 * benchmark's roofline figure.  Enabled by apic_set_profiling. */
typedef struct {
  int64_t steps;
  int64_t iter_launches;   /* launches of the fused transfer kernel           */
  double iter_ms;          /* their summed durations                           */
  double prep_ms;          /* keys, sort, gather, grid activation, up to the
                              host's read of the grid size                     */
  double step_ms;          /* whole steps                                      */
  int64_t particles;       /* particles of the last step                      */
  int64_t active_nodes;    /* grid nodes of the last step                     */
  int64_t kernel_launches; /* launches of this library's own kernels          */
  int64_t sort_launches;   /* device sort / scan primitive calls (CUB)        */
  double mass_ms;          /* mass + P2G(V) pass, friction blend, normalise    */
  int64_t graph_launches;  /* CUDA graph launches (sizing and series regions) */
} apic_profile;

/* Bounds checks of the kernels' own indexing (not in the paper).  A library
 * built with -DAPIC_DEBUG_BOUNDS (libapiccontact_debug.so) checks tile-node,
 * page-table, particle-slot, permutation and sort-output indices on the
 * device; a failed check records a bit and skips the access (no trap).
 * apic_debug_build returns 1 for such a library, 0 otherwise;
 * apic_debug_flags returns the recorded bits (1 tile node, 2 page-table
 * index, 4 item size or cell bits, 8 permutation entry, 16 sort output
 * position) of the current device, 0 in the normal build, and clears them
 * when `clear` is non-zero. */
int32_t apic_debug_build(void);
apic_status apic_debug_flags(uint32_t* out, int32_t clear);

/* Message of the last failed call on this thread ("" if none). */
const char* apic_last_error(void);

/* Library version string. */
const char* apic_version(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the
 * scratch the context may hold (0 = no cap).  Returns INVALID_ARG for a bad
 * device, CUDA on a runtime failure. */
apic_status apic_create(apic_ctx** out, int32_t device, size_t hbm_budget_bytes);

/* Free a context and all its scratch.  NULL is accepted. */
apic_status apic_destroy(apic_ctx* ctx);

/* One contact step (Sec. 2.3 series with the Sec. 2.4 projection).
 * Asynchronous on `stream` except for these host synchronisations of the
 * stream:
 *   - while sizing the sparse grid: once when the context reuses the
 *     page-table box of its previous step (the steady state of a
 *     simulation), twice when a box must be fitted (the first step, or a
 *     particle that left the reused box);
 *   - at the end when `stats` is non-NULL or APIC_HOST_PTRS is set;
 *   - with APIC_DETERMINISTIC, once more after the series to read the
 *     fixed-point range flags, and, if a range was exceeded, a second run of
 *     the series followed by one more synchronisation.
 * Invalid particle data (body out of range, m <= 0, non-finite or
 * out-of-range positions) returns INVALID_ARG. */
apic_status apic_contact_step(apic_ctx* ctx, const apic_step_args* args, void* stream, apic_stats* stats);

/* Several independent scenes in one call (Sec. 2.3 series on each).
 * Each scene keeps its own particles, grid spacing h, friction (mu or
 * mu_pair) and outputs; the scenes share one sort, one sparse page table
 * and one launch per transfer pass over the flattened work list, so small
 * scenes fill the GPU together.  All scenes must share `flags` and
 * `n_iter`.  `stats` is NULL or an array of n_scenes entries.  Host or
 * device pointers, synchronisation and errors as apic_contact_step; an error
 * message names the offending scene. */
apic_status apic_contact_step_batched(apic_ctx* ctx, const apic_step_args* scenes, int32_t n_scenes,
                                      void* stream, apic_stats* stats);

/* Normals from each body's grid mass, for callers with neither normals nor
 * a surface mesh (the paper's normals come from the FE surface, Sec. 2.3;
 * this construction is the library's): for particle p of body b,
 *   rho_p = sum_i N_i(x_p) m_{b,i},   g_p = sum_i grad N_i(x_p) m_{b,i}
 * with m_{b,i} body b's grid mass (eq. massToGrid over body b alone, App. B
 * weights), and nrm_out[p] = -g_p / |g_p| where |g_p| h > threshold * rho_p,
 * else 0.  threshold 0.5 is what APIC_MASS_NORMALS uses.
 *   args     the scene as for apic_contact_step: n, n_bodies, body, x, m, h
 *            and flags are read (APIC_FP64 and APIC_DETERMINISTIC only);
 *            v, C, nrm, v_out, C_out, mu, mu_pair and n_iter are ignored.
 *   nrm_out  [n*3] DEVICE array (float, or double with APIC_FP64), written
 *            in the caller's particle order.
 * Device pointers only; asynchronous on `stream` except for the host
 * synchronisations of the grid sizing (see apic_contact_step).  Invalid
 * positions, masses or body ids return INVALID_ARG. */
apic_status apic_mass_normals(apic_ctx* ctx, const apic_step_args* args, double threshold, void* nrm_out,
                              void* stream);

/* The contact step for callers that cannot allocate device memory.
 * (The paper has no counterpart; this is a deployment variant.)
 *
 * Some hosts may not call cudaMalloc during a step: an application whose own
 * memory pool has already reserved (nearly) all of the GPU and hands out
 * nothing else, or a real-time loop that cannot afford the device-wide
 * synchronisation cudaMalloc and cudaFree imply.  This call computes the
 * same contact step as apic_contact_step, on the same apic_step_args and
 * apic_stats (within floating-point rounding: it always runs the default
 * kernel variant with direct launches; with APIC_DETERMINISTIC the bits are
 * identical), but takes every scratch buffer from one static device array of
 * 32 MiB that the library defines (one per GPU that loads the library, held
 * until the process exits).  It allocates nothing and needs no context.
 *   - Device pointers only (APIC_HOST_PTRS is rejected).
 *   - A scene whose scratch would exceed the 32 MiB array (roughly 100,000
 *     FP32 particles in compact bodies; fewer for sparse scenes or FP64) is
 *     rejected with APIC_ERR_INVALID_ARG and a message naming the limit.
 *   - The array belongs to the current device (cudaGetDevice): make the
 *     device of the arrays and the stream current before the call.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress; nothing is cached, so a device reset does not
 *     leave a stale address).  The first call on a device loads the
 *     library's device code there; make that first call before any stream
 *     capture begins.
 *   - Every call uses the same array and leaves its data there; each call
 *     clears what must start at zero.  Calls whose GPU work overlaps (other
 *     streams, other host threads) race on the array: serialise them.
 *   - Synchronises the stream twice while sizing the grid (there is no
 *     page-table box to reuse between calls), and at the end when stats is
 *     non-NULL; with APIC_DETERMINISTIC once more after the series, and, if
 *     a fixed-point range was exceeded, after a second run of the series.
 *     Errors are reported by apic_last_error(). */
apic_status apic_contact_step_static(const apic_step_args* args, void* stream, apic_stats* stats);

/* ---------------------------------------------------------------------------
 * Serving: many concurrent simulations, state resident on the device.
 *
 * A server owns worker threads, each with its own context and CUDA stream.
 * A simulation (apic_sim) keeps its particles' x, v, C, m, normals and body
 * ids on the device between steps.  apic_sim_submit queues one contact step
 * of that simulation (the step writes V_hat back into v and C, then, when
 * dt_advect > 0, moves x += dt_advect * v).  Workers take every ready request
 * (at most one in flight per simulation, FIFO per simulation) and run them
 * as one batched step; a request that arrives while a batch is on the GPU is
 * picked up by the next free worker, so batches overlap on the device.
 * Requests are batched only with requests of the same flags and n_iter.
 * Unlike a context, a server may be called from any host thread (every call
 * takes the server's lock).  The paper steps one simulation at a time; this
 * serving layer has no counterpart in it.
 * --------------------------------------------------------------------------*/
typedef struct apic_server apic_server;
typedef struct apic_sim apic_sim;

typedef struct {
  int64_t completed;        /* completed step requests                       */
  int64_t failed;           /* requests that ended in an error               */
  int64_t batches;          /* batched launches                              */
  int64_t particle_iters;   /* sum of n * (n_iter + 1) over completed steps  */
  double latency_p50_ms;    /* submit -> completion, over completed requests */
  double latency_p99_ms;
  double latency_mean_ms;
  double mean_batch_scenes; /* requests per batched launch                   */
  int64_t resident_bytes;   /* device bytes held by open simulations         */
  int64_t open_sims;
} apic_server_stats;

/* Create a server on `device` with `n_workers` worker threads (>= 1).
 * hbm_budget_bytes caps the resident state of open simulations plus the
 * workers' scratch (0 = no cap); max_batch_scenes caps requests per batch. */
apic_status apic_server_create(apic_server** out, int32_t device, size_t hbm_budget_bytes, int32_t n_workers,
                               int32_t max_batch_scenes);

/* Launch policy of the workers' contexts for the batches they start from now
 * on: `variant` as apic_set_variant (-1: tune per size class, the default),
 * `graphs` as apic_set_graphs (1, the default).  Not in the paper. */
apic_status apic_server_set_policy(apic_server* srv, int32_t variant, int32_t graphs);

/* Finish queued requests, stop the workers, free every simulation. */
apic_status apic_server_destroy(apic_server* srv);

/* Admit a simulation: copy its state (host or device pointers per
 * APIC_HOST_PTRS) to resident device memory.  h, mu, mu_pair, n_iter and
 * flags are kept for its steps; v_out / C_out are ignored.  Returns
 * APIC_ERR_ADMISSION when the budget cannot hold it now (retry after other
 * simulations close). */
apic_status apic_sim_open(apic_server* srv, const apic_step_args* init, apic_sim** out);

/* Queue one contact step of `sim`; *ticket identifies the request. */
apic_status apic_sim_submit(apic_sim* sim, double dt_advect, uint64_t* ticket);

/* Has the request finished?  done = 1 and its latency (submit -> completion)
 * when it has; returns the request's own error status if it failed.  A
 * finished request is forgotten once reported (here or by apic_ticket_wait),
 * and when its simulation closes: later queries of it return
 * APIC_ERR_INVALID_ARG ("unknown ticket"). */
apic_status apic_ticket_poll(apic_server* srv, uint64_t ticket, int32_t* done, double* latency_ms);

/* Wait at most timeout_s seconds for the request; APIC_ERR_TIMEOUT if it has
 * not finished by then (the request stays known).  Once it returns after the
 * request finished, the ticket is forgotten, as for apic_ticket_poll. */
apic_status apic_ticket_wait(apic_server* srv, uint64_t ticket, double timeout_s, double* latency_ms);

/* Copy the simulation's current state to HOST memory (each pointer may be
 * NULL): x [n*3] doubles, v [n*3] and C [n*9] in the simulation's precision.
 * Waits for its queued and running steps first. */
apic_status apic_sim_read(apic_sim* sim, double* x_out, void* v_out, void* C_out);

/* Checkpoint: the simulation's whole state (positions, body ids, v, C, masses,
 * normals, h, mu, mu_pair, n_iter, flags) into a HOST buffer, after its queued
 * and running steps.  With host_buf NULL, *bytes receives the size needed;
 * otherwise *bytes is the buffer's size on entry (APIC_ERR_INVALID_ARG if too
 * small) and the size written on return.  The format is this library's own,
 * in host byte order. */
apic_status apic_sim_export(apic_sim* sim, void* host_buf, size_t* bytes);

/* Resume: open a new simulation on srv from a checkpoint written by
 * apic_sim_export (admission as apic_sim_open).  APIC_ERR_INVALID_ARG for a
 * buffer that is not a complete checkpoint of this library. */
apic_status apic_sim_import(apic_server* srv, const void* host_buf, size_t bytes, apic_sim** out);

/* ---------------------------------------------------------------------------
 * Server groups: simulations spread over several devices by HBM budget.
 * (Not in the paper.)  Simulations are independent, so a group is one
 * server per device and nothing crosses devices on the data path: a
 * simulation lives on the device it was admitted to, and its requests, tickets
 * and reads go to that device's server (apic_sim_server).
 * --------------------------------------------------------------------------*/
typedef struct apic_group apic_group;

/* The device (index into free_bytes) with the most room that still holds
 * `need` bytes (ties: the lowest index), or -1 when none does.  free_bytes
 * of a device without a budget is INT64_MAX.  Host function, no GPU. */
int32_t apic_place_by_budget(const int64_t* free_bytes, int32_t n_devices, int64_t need);

/* One server per listed device (the same device may be listed twice: two
 * independent servers), each with hbm_budget_per_device (0 = no cap),
 * n_workers workers and max_batch_scenes as apic_server_create. */
apic_status apic_group_create(apic_group** out, const int32_t* devices, int32_t n_devices,
                              size_t hbm_budget_per_device, int32_t n_workers, int32_t max_batch_scenes);

/* Destroy every member server (finishing queued requests first). */
apic_status apic_group_destroy(apic_group* group);

/* Member `member` (0..n_devices-1) of the group. */
apic_status apic_group_server(apic_group* group, int32_t member, apic_server** out);

/* apic_server_set_policy on every member. */
apic_status apic_group_set_policy(apic_group* group, int32_t variant, int32_t graphs);

/* Admit a simulation on the member with the most room for it
 * (apic_place_by_budget over each member's budget minus its resident state
 * and worker scratch); *member (may be NULL) receives the member's index.
 * A member that refuses because others were admitted meanwhile is skipped;
 * APIC_ERR_ADMISSION when no member has room now. */
apic_status apic_group_open(apic_group* group, const apic_step_args* init, apic_sim** out, int32_t* member);

/* Statistics summed over the members; latency percentiles over all of their
 * samples. */
apic_status apic_group_get_stats(apic_group* group, apic_server_stats* out, int32_t reset);

/* The server that holds `sim` (for its tickets). */
apic_status apic_sim_server(apic_sim* sim, apic_server** out);

/* Wait for the simulation's steps, then free its resident state. */
apic_status apic_sim_close(apic_sim* sim);

/* Counters and latency percentiles since creation (or the last reset); the
 * percentiles cover at most the last 2^20 completed requests. */
apic_status apic_server_get_stats(apic_server* srv, apic_server_stats* out, int32_t reset);

/* Diagnostics (no counterpart in the paper). */

/* Turn kernel timing on (1) or off (0) and reset the counters. */
apic_status apic_set_profiling(apic_ctx* ctx, int32_t on);

/* Read the counters (synchronises the device work they cover). */
apic_status apic_get_profile(apic_ctx* ctx, apic_profile* out);

/* Bytes of device scratch the context currently holds. */
apic_status apic_scratch_bytes(apic_ctx* ctx, size_t* out);

/* Node normals n_p for apic_step_args.nrm, built as Sec. 2.3 builds them:
 * the outward normals of the boundary faces adjacent to each node, weighted
 * by face area, summed and normalised.
 *   x    [n*3] node positions (doubles, AoS xyz), the configuration the
 *        normals are wanted in;
 *   tri  [n_tri*3] int32 node ids of the boundary triangles, each wound
 *        counter-clockwise seen from outside (split quads into two); NULL
 *        when n_tri = 0;
 *   nrm_out [n*3] unit normals, float (or double with APIC_FP64); 0 for a
 *        node on no triangle (interior nodes) or on zero-area ones only.
 * Flags: APIC_FP64, APIC_HOST_PTRS (all three arrays in host memory).  The
 * sums are FP64 (atomic, so their rounding order varies between calls, far
 * below FP32 resolution).  Scratch (24 bytes per node, plus staging for host
 * arrays) comes from the context.  Synchronises `stream` before returning;
 * APIC_ERR_INVALID_ARG if a triangle index is outside [0, n) (nrm_out is then
 * unspecified). */
apic_status apic_node_normals(apic_ctx* ctx, int64_t n, const double* x, int64_t n_tri, const int32_t* tri,
                              void* nrm_out, uint32_t flags, void* stream);

/* ---------------------------------------------------------------------------
 * Augury dynamics (Sec. 2.2): the contact step inside a time integrator.
 *
 * eq. apic_accel gives the contact acceleration A_hat = (H - I) V_bar / tau of
 * the predicted generalized velocity V_bar = V_t + tau A_t; eq. apic_Augury
 * adds it to the mechanical acceleration; eq. Newmark integrates.  The printed
 * eq. Newmark has garbled half-step indices; it is read as velocity Verlet:
 *   V^{n+1/2} = V^n + dt/2 A^n;  x^{n+1} = x^n + dt v^{n+1/2};
 *   A^{n+1} = {a(x^{n+1}), 0} + A_hat^{n+1};  V^{n+1} = V^{n+1/2} + dt/2 A^{n+1},
 * with V_t = V^{n+1/2} + dt/2 {a(x^{n+1}), 0} (the velocity at t^{n+1} before
 * contact).  H is apic_contact_step on normals rebuilt every step from the
 * boundary triangles (apic_node_normals).  The mechanical acceleration comes
 * from linear springs (a stand-in for the paper's finite elements, which are
 * out of scope) plus uniform gravity.  Not a paper listing: the paper gives
 * the equations, not this API.
 * --------------------------------------------------------------------------*/
#define APIC_AUGURY_INIT (1u << 4) /* first compute A^0 at x^0 (V_t = V^0) */

typedef struct {
  int64_t n;                 /* nodes (particles), > 0                               */
  int32_t n_bodies;          /* as apic_step_args                                    */
  int32_t n_iter;            /* N of the contact step                                */
  const int32_t* body;       /* [n]                                                  */
  double* x;                 /* [n*3] positions, advanced in place                   */
  void* v;                   /* [n*3] velocity, advanced in place (float; double with APIC_FP64) */
  void* C;                   /* [n*9] affine velocity C = B D^-1, advanced in place   */
  void* av;                  /* [n*3] acceleration A^n (v part), carried between calls */
  void* aC;                  /* [n*9] acceleration A^n (C part)                      */
  const void* m;             /* [n] masses > 0                                       */
  const uint8_t* fixed;      /* [n] nonzero: node held (v = C = A = 0), or NULL       */
  int64_t n_springs;         /* linear springs between node pairs                    */
  const int32_t* springs;    /* [n_springs*2] node ids                               */
  const double* rest;        /* [n_springs] rest lengths                             */
  const double* stiffness;   /* [n_springs] spring constants (force per length)      */
  double gravity[3];         /* uniform acceleration                                 */
  int64_t n_tri;             /* boundary triangles for the normals (0: all normals 0) */
  const int32_t* tri;        /* [n_tri*3], outward winding                           */
  double h, mu;              /* grid spacing, friction (as apic_step_args)           */
  const double* mu_pair;     /* host, n_bodies^2, or NULL                            */
  double dt, tau;            /* time step and augury time (the paper uses tau = dt)  */
  uint32_t flags;            /* APIC_FP64, APIC_VARIANT_PIC, APIC_VARIANT_SEP23, APIC_AUGURY_INIT */
} apic_augury_args;

typedef struct {
  double P[3], L[3];         /* linear and angular momentum (L with the affine spin term) */
  double kinetic;            /* sum 1/2 m |v|^2                                      */
  double springs;            /* sum 1/2 k (|d| - L0)^2                               */
  double gravity;            /* -sum m g.x                                           */
} apic_augury_stats;

/* Advance the state n_steps time steps on `stream` (device pointers only).
 * Scratch comes from the context.  Synchronises before returning.  Errors:
 * APIC_ERR_INVALID_ARG for bad sizes, NULL arrays, disallowed flags, or a
 * spring or triangle index outside [0, n) (the state is then unspecified);
 * the contact step's own errors pass through.  stats (nullable) describe the
 * final state. */
apic_status apic_augury_steps(apic_ctx* ctx, const apic_augury_args* args, int32_t n_steps, void* stream,
                              apic_augury_stats* stats);

/* ---------------------------------------------------------------------------
 * Kernel variants, autotuning and CUDA graphs (no counterpart in the paper:
 * they change how the transfer passes are launched, never what they compute).
 *
 * The fused transfer kernel is built in apic_variant_count() variants that
 * differ in how many 128-thread CTAs each SM holds (register cap versus
 * occupancy); which is fastest depends on the scene.  By default a context
 * tunes per size class (FP32 path; classes = bit length of the call's total
 * particle count): the first calls of a class run each variant twice, timed
 * with CUDA events on the caller's stream, and the fastest is used from then
 * on.  The FP64 path has one variant.
 *
 * The launch sequence from the mass pass to the last transfer pass is
 * captured as a CUDA graph on the second consecutive call whose sizes and
 * buffers match the previous call's, and replayed while they keep matching.
 * --------------------------------------------------------------------------*/

/* Number of variants, and a one-line description of variant v ("" if out of
 * range; the string is static). */
int32_t apic_variant_count(void);
const char* apic_variant_name(int32_t v);

/* Fix the variant for every later call on ctx (0 .. count-1), or -1 to tune
 * per size class (the default).  APIC_ERR_INVALID_ARG if out of range. */
apic_status apic_set_variant(apic_ctx* ctx, int32_t v);

/* The variant used for a call of n_particles FP32 particles: *decided = 1 and
 * the tuned (or fixed) variant, or *decided = 0 and variant 0 while the size
 * class is still being tuned. */
apic_status apic_get_variant(apic_ctx* ctx, int64_t n_particles, int32_t* variant, int32_t* decided);

/* Tune the size class of these scenes now: runs apic_contact_step_batched on
 * them until the class is decided (at most 2 * count + 1 calls, synchronising
 * `stream` after each) and returns the choice in *variant (nullable).  The
 * outputs are overwritten by every call; with in-place arrays (v_out == v)
 * the state advances, so tune on a copy.  APIC_ERR_INVALID_ARG when a variant
 * is fixed. */
apic_status apic_autotune(apic_ctx* ctx, const apic_step_args* scenes, int32_t n_scenes, void* stream,
                          int32_t* variant);

/* The autotuner's decisions, to keep across processes (e.g. in a file keyed
 * by the GPU model): *count = the number of decided size classes (the FP32
 * particle count's bit length); the first min(count, cap) go to classes[] and
 * variants[].  apic_set_tuning marks the given classes decided with the given
 * variants (no timing); APIC_ERR_INVALID_ARG for a class outside [0, 62] or a
 * variant outside [0, apic_variant_count()), and then nothing is set.  Not in
 * the paper. */
apic_status apic_get_tuning(apic_ctx* ctx, int32_t* classes, int32_t* variants, int32_t cap, int32_t* count);
apic_status apic_set_tuning(apic_ctx* ctx, const int32_t* classes, const int32_t* variants, int32_t count);

/* Capture and replay the transfer passes as a CUDA graph (1, the default) or
 * launch them one by one (0).  Profiling (apic_set_profiling) launches them
 * one by one regardless, to time each pass. */
apic_status apic_set_graphs(apic_ctx* ctx, int32_t on);

/* Device memory for the context's scratch (sort buffers, sorted particle
 * planes, grid nodes, staging) from the caller's allocator instead of
 * cudaMalloc, e.g. a framework's caching allocator.  alloc(user, bytes,
 * device) returns a device pointer aligned to 256 bytes, or NULL (the call
 * that needed it fails with APIC_ERR_OUT_OF_MEMORY); free(user, ptr, bytes,
 * device) takes back a block alloc returned.  The library synchronises the
 * device before it hands a block back (scratch grows rarely, and a caching
 * allocator may reuse the block at once) and frees everything in
 * apic_destroy.  The budget of apic_create still applies.  Give both
 * functions, or neither (cudaMalloc); set them before the first step:
 * APIC_ERR_INVALID_ARG once the context holds scratch.  Small fixed buffers
 * (device counters, page-locked staging tables) stay the library's.  Not in
 * the paper. */
typedef void* (*apic_alloc_fn)(void* user, size_t bytes, int32_t device);
typedef void (*apic_free_fn)(void* user, void* ptr, size_t bytes, int32_t device);
apic_status apic_set_allocator(apic_ctx* ctx, apic_alloc_fn alloc, apic_free_fn free_fn, void* user);

/* Launch each transfer pass and node normalisation with programmatic
 * dependent launch (1, the default), so that a grid's prologue overlaps the
 * end of the grid before it, or strictly one after another (0).  The results
 * are the same either way.  Profiling launches them strictly in order. */
apic_status apic_set_overlap(apic_ctx* ctx, int32_t on);

#ifdef __cplusplus
}
#endif

#endif /* APICCONTACT_H */
