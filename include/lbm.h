/*
 * liblbm -- GB300 (sm_103a) fused streaming + MRT collision step of the
 * incompressible 14- and 18-velocity lattice Boltzmann models of
 * Zhang, Shi & Wang, "Incompressible MRT lattice Boltzmann models in three
 * dimensions" (arXiv:1503.03337).
 *
 * Problem statement (Sec. 4): a box of nx*ny*nz fluid nodes; every face is
 * periodic, a no-slip wall or a moving wall; viscosity nu (Eq. vis); an
 * optional body force; output velocity u and pressure p (Eq. hgl).
 *
 * Conventions shared by every call:
 *  - Nodes are ordered x fastest: cell = x + nx*(y + ny*z).
 *  - Population arrays are [a][cell], a = 0..Q-1 being the paper's direction
 *    a+1 (Sec. 3 velocity set for Q = 14, App. B for Q = 18).  Q = 26 is
 *    the D3Q27 set without c_0 that App. B's closing remark names: the 18
 *    directions of Q = 18 in their order, then the 8 cube diagonals in the
 *    order of Q = 14's directions 7..14.
 *  - Walls sit halfway between the last fluid node and the ghost node beyond
 *    it (halfway bounce-back); a moving wall adds 6 w_a (c_a . u_wall) to the
 *    reflected population.
 *  - Lattice units throughout (dx = dt = c = 1, c_s^2 = 1/3).
 *  - Every call returns LBM_OK (0) or one of the LBM_E* codes below; no C++
 *    exception crosses this boundary.  lbm_last_error() gives a message for
 *    the calling thread's last failure.
 *  - A handle is not thread-safe: one handle per host thread, or external
 *    locking.  All GPU work of a handle is queued on the stream it was given.
 *  - Device pointers passed in must be on the handle's device; host pointers
 *    may be pageable or pinned.  The caller keeps ownership of every buffer
 *    it passes; the library never frees a caller's buffer.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define LBM_OK 0
#define LBM_EINVAL 1    /* bad argument, size or state                       */
#define LBM_ENOMEM 2    /* device or pinned host allocation failed          */
#define LBM_ECUDA 3     /* a CUDA runtime call or kernel launch failed      */
#define LBM_EUNSTABLE 4 /* a reduction found a non-finite velocity          */
#define LBM_ETIMEOUT 5  /* a bounded device-side wait gave up               */
#define LBM_EBUSY 6     /* no free slot / memory budget exhausted           */

/* ---- enumerations ------------------------------------------------------- */
enum lbm_storage { /* how populations are held in device memory */
  LBM_STORAGE_F64 = 0,  /* double; all arithmetic in double (parity build) */
  LBM_STORAGE_F32 = 1,  /* float; arithmetic in float                      */
  LBM_STORAGE_F16 = 2,  /* IEEE half; arithmetic in float                   */
  LBM_STORAGE_BF16 = 3  /* bfloat16; arithmetic in float                    */
};

enum lbm_face_kind {
  LBM_PERIODIC = 0,    /* wraps to the opposite face (both must say so)   */
  LBM_WALL = 1,        /* halfway bounce-back, wall at rest               */
  LBM_MOVING_WALL = 2, /* halfway bounce-back with wall velocity u_wall   */
  LBM_SYMMETRY = 3,    /* free-slip mirror plane halfway beyond the face:
                        * a population leaving through it returns as its
                        * mirror image (normal velocity component
                        * reversed) at the node it left.  Where a link also
                        * crosses a wall face the wall's bounce-back
                        * applies.  Like a wall, it cannot face a periodic
                        * face.  Sec. 4.3's reduced domains use it. */
  /* Non-equilibrium extrapolation, the boundary scheme of Sec. 4 (after
   * Guo, Zheng and Shi): the outermost node layer lies ON the face.  After
   * every step each node x_b of such a layer takes
   *   f(x_b) = f_eq(p_b, u_b) + [f(x_f) - f_eq(p_f, u_f)]   (Eq. edf),
   * x_f being its neighbour one node inward along the normal of every such
   * face it lies on (diagonally inward on edges and corners) and (p_f, u_f)
   * the macroscopic values there (Eq. hgl).  u_b is prescribed on a
   * velocity face (u_wall of the first such face in x-, x+, y-, y+, z-, z+
   * order), else u_b = u_f; p_b is prescribed on a pressure face
   * (lbm_params.p_face of the first such face), else p_b = p_f, so a node
   * where a wall meets an inlet takes u_wall and the inlet pressure.  The
   * axis of such a face needs at least 3 nodes. */
  LBM_NEQ_VELOCITY = 4,
  LBM_NEQ_PRESSURE = 5
};

enum lbm_face { LBM_XM = 0, LBM_XP = 1, LBM_YM = 2, LBM_YP = 3, LBM_ZM = 4, LBM_ZP = 5 };

enum lbm_field_bits {
  LBM_FIELD_U = 1u,          /* 3*N values: ux[N], uy[N], uz[N]            */
  LBM_FIELD_P = 2u,          /* N values                                   */
  LBM_FIELD_POPULATIONS = 4u /* Q*N values, canonical pre-collision f^n    */
};

enum lbm_dtype { LBM_DTYPE_F64 = 0, LBM_DTYPE_F32 = 1 };

/* Rounding of FP16/BF16 stores (ignored for FP32/FP64 storage).  Nearest
 * loses every per-step change below half a storage ulp in the same
 * direction; stochastic rounding makes each store unbiased: the value goes
 * to the 16-bit neighbour above with probability equal to its distance from
 * the one below, over their spacing, quantised to 13 (FP16) or 16 (BF16)
 * random bits from a counter-based hash of (cell pair, direction, step), so
 * runs are reproducible and independent of launch shape and batching. */
enum lbm_rounding { LBM_ROUND_NEAREST = 0, LBM_ROUND_STOCHASTIC = 1 };

/* ---- descriptors -------------------------------------------------------- */
typedef struct lbm_desc {
  int32_t Q;       /* 14 (Sec. 3), 18 (App. B) or 26 (App. B's closing
                      remark: the same construction on D3Q27 without c_0;
                      single-domain handles only)                         */
  int32_t nx, ny, nz; /* fluid nodes per axis, each >= 1                   */
  int32_t storage; /* enum lbm_storage                                     */
} lbm_desc;

/* Face order x-, x+, y-, y+, z-, z+.  A ghost node beyond several faces
 * (an edge or corner) takes the velocity of the first MOVING_WALL face among
 * them in that order, else zero.
 *
 * Edge profile of a MOVING_WALL face f (the lid corner velocities of Sec.
 * 4.3): edge_axis[f] = k + 1 names an in-plane axis k of the face; the
 * wall velocity seen from the first node column along k is
 * u_wall[f] * edge_scale[f][0], from the last one u_wall[f] *
 * edge_scale[f][1] (a one-node axis takes [0]), elsewhere u_wall[f].
 * edge_axis[f] = 0 (a zero-initialised struct) leaves the face uniform.
 * LBM_EINVAL: edge_axis outside 0..3, on a face that is not a moving wall,
 * along the face's normal, or a non-finite scale. */
typedef struct lbm_geom {
  int32_t face[6];
  double u_wall[6][3];
  int32_t edge_axis[6];
  double edge_scale[6][2];
} lbm_geom;

/* Relaxation rates of the diagonal collision matrix, Eq. sD3Q15meaning
 * (Q14) and Eq. sD3Q19 (Q18).  If nu > 0 then s_nu = 1/(3 nu + 1/2)
 * (Eq. vis) and the s_nu field is ignored.  Sec. 4 uses s_c = 1, s_e = 1.19,
 * s_q = 1.2, s_t = 0.98; s_pi (Q18 and Q26) is not given by the paper.
 * Q26 (no rates in the paper) gives each of its rows beyond the 18 of Q18
 * the rate of the Q18 row it extends: |c|^4 s_e, the |c|^4 c rows s_q, the
 * |c|^2 c_x c_y rows s_pi, c_x c_y c_z s_t.
 * Body force F(t_n) = force * cos(2 pi n / force_period) if force_period > 0,
 * else force; it enters as u = j + F/2 and a Guo source in moment space.
 * p_ref shifts the reported pressure: stored populations are
 * f_a - 3 w_a p_ref, and read-back p includes p_ref. */
typedef struct lbm_params {
  double nu;
  double s_nu, s_c, s_e, s_q, s_pi, s_t;
  double force[3];
  double force_period;
  double p_ref;
  int32_t residual_interval; /* > 0: lbm_step runs the FP64 reductions every
                                that many steps (stats via lbm_read_stats) */
  int32_t rounding;          /* enum lbm_rounding */
  /* Pressure of each LBM_NEQ_PRESSURE face at time level n:
   * p_face[f] + p_amp[f] * cos(2 pi n / p_period) if p_period > 0, else
   * p_face[f] (Sec. 4.1 constant inlet/outlet pressures; Sec. 4.2
   * oscillating pressure drop, Eq. pbc-pul).  Same units as the read-back
   * pressure (p_ref included). */
  double p_face[6];
  double p_amp[6];
  double p_period;
} lbm_params;

/* FP64 reductions over all nodes at step `step`, against the velocity
 * snapshot of step `prev_step` (-1: none yet).  They give the convergence
 * criteria of Eq. sc, Eq. cr and Eq. cavity_creterion:
 *   sc     = sum_abs_du[k] / sum_abs_u_prev[k]   (one component k)
 *   cr     = sum_abs_du[k] / sum_abs_u[k]
 *   cavity = sum_k sum_abs_du[k] / sum_k sum_abs_u[k]. */
typedef struct lbm_stats {
  int64_t step, prev_step;
  double sum_abs_du[3];
  double sum_abs_u[3];
  double sum_abs_u_prev[3];
  double sum_P;     /* sum of P = sum_a f_a (mass-like invariant)        */
  double sum_u[3];  /* sum of u (volume flux)                            */
  double max_abs_u; /* largest |u_k| over nodes and components          */
  int64_t nonfinite;/* nodes whose P or u is not finite                  */
} lbm_stats;

typedef struct lbm_handle lbm_handle;

/* ---- single domain ------------------------------------------------------ */

/* Allocate a domain on the current CUDA device: one population buffer of
 * Q*nx*ny*nz storage values (single-buffer AA streaming) plus a small
 * reduction workspace.  `cuda_stream` is a cudaStream_t (NULL = legacy
 * default stream); it is borrowed, not owned.  Initial state: all walls at
 * rest, Sec. 4 default rates with nu = 1/6, no force, f = 0, step 0.
 * Domains of up to 2^31 - 1 cells (D3Q18 FP32: 154 GB); where Q*N >= 2^31
 * the step runs one cell per thread with 64-bit population offsets
 * (cells_per_thread = 2 is accepted and has no effect there).
 * Errors: EINVAL (Q not 14/18/26, a size < 1, storage unknown,
 * nx*ny*nz >= 2^31, nz > 65535),
 * ENOMEM, ECUDA. */
int lbm_create(const lbm_desc *desc, void *cuda_stream, lbm_handle **out);

/* Free everything the handle owns.  NULL is accepted. */
void lbm_destroy(lbm_handle *h);

/* Replace the stream later work is queued on. */
int lbm_set_stream(lbm_handle *h, void *cuda_stream);

/* Boundary kinds (Sec. 4 problem statement): halfway and moving-wall
 * bounce-back, symmetry planes, or the paper's own non-equilibrium
 * extrapolation (LBM_NEQ_*).  EINVAL if a kind is unknown, only one of two
 * opposite faces is periodic, or an LBM_NEQ_* face lies on an axis with
 * fewer than 3 nodes, or LBM_NEQ_* faces while a solid mask is set. */
int lbm_set_geometry(lbm_handle *h, const lbm_geom *geom);

/* Rates, force and reduction cadence.  EINVAL unless every rate is in
 * (0, 2), nu > 0 or s_nu given, and all values are finite. */
int lbm_set_params(lbm_handle *h, const lbm_params *params);

/* Solid nodes (general geometry; the paper's introduction motivates complex
 * boundaries and porous media): `solid` holds N bytes, x fastest, nonzero
 * marking a solid node (host pointer, or device if on_device != 0; copied,
 * the caller keeps it).  A fluid node whose pull source is solid -- after
 * the periodic wraps and symmetry mirrors of the faces -- bounces that
 * population back as off a wall at rest halfway between the two nodes.
 * Solid nodes hold no flow: no step updates them, lbm_read_fields reports
 * zero there, lbm_reductions leaves them out, lbm_write_populations
 * ignores their values.  NULL returns to the plain box.  Set it before
 * lbm_init_equilibrium (or restore a checkpoint after it): the populations
 * of a node that turns solid or fluid are not converted.  Costs N*5 bytes
 * of device memory and 4 bytes of traffic per cell update; two cells per
 * thread is not used while a mask is set.  Not for handles with
 * LBM_NEQ_* faces.  Synchronises.  EINVAL, ENOMEM, ECUDA. */
int lbm_set_solid(lbm_handle *h, const uint8_t *solid, int on_device);

/* f = f_eq(p, u) of Eq. edf at every node (u: 3*N FP64 ux,uy,uz; p: N FP64;
 * either may be NULL meaning zero), step counter reset to 0, velocity
 * snapshot cleared.  Pointers are device pointers if on_device != 0. */
int lbm_init_equilibrium(lbm_handle *h, const double *u, const double *p, int on_device);

/* Queue nsteps fused steps (stream + collide, Eq. mrteqvT) on the stream.
 * Asynchronous.  Returns LBM_EUNSTABLE without queuing anything if an
 * earlier reduction found non-finite values (until the next init or
 * write_populations). */
int lbm_step(lbm_handle *h, int64_t nsteps);

/* Current step counter n (populations hold f^n). */
int lbm_get_step(lbm_handle *h, int64_t *n);

/* Set the step counter to n >= 0 without touching device memory (the force
 * time level and the parity of the storage layout follow n).  Meant to be
 * followed by lbm_write_populations when restoring a checkpoint taken at
 * step n.  Clears the velocity snapshot. */
int lbm_set_step(lbm_handle *h, int64_t n);

/* Copy the fields selected by `mask` (LBM_FIELD_* bits), in the order U, P,
 * POPULATIONS, back to back, into dst as FP64 or FP32 (dtype).  u is
 * j + F(t_n)/2, p follows Eq. hgl plus p_ref.  Synchronises the stream. */
int lbm_read_fields(lbm_handle *h, unsigned mask, void *dst, int dst_on_device, int dtype);

/* Overwrite the state with canonical pre-collision populations (Q*N FP64)
 * at the current step counter (checkpoint restore).  Synchronises. */
int lbm_write_populations(lbm_handle *h, const double *src, int src_on_device);

/* Run the FP64 reductions now (current populations against the last
 * snapshot), make the current velocity the new snapshot, and return the
 * statistics.  Synchronises.  With FP64 storage the arithmetic is FP64;
 * with FP32/FP16/BF16 storage it runs on pairs of FP32 numbers (about 48
 * significant bits, combined in FP64 at the end), whose results agree with
 * FP64 sums of the fields to about 1e-13 relative. */
int lbm_reductions(lbm_handle *h, lbm_stats *out);

/* Statistics of the most recent reduction (queued by lbm_step's cadence or
 * lbm_reductions).  Synchronises. */
int lbm_read_stats(lbm_handle *h, lbm_stats *out);

/* Convergence criteria of the paper, formed from one lbm_stats (the sums of
 * a reduction at step t1 = s->step against the snapshot of t0 =
 * s->prev_step):
 *   LBM_RESIDUAL_STEADY   Eq. sc (Sec. 4.1), one velocity component k:
 *       sum_i |u_k(t1) - u_k(t0)| / sum_i |u_k(t0)|   (earlier level)
 *   LBM_RESIDUAL_PERIODIC Eq. cr (Sec. 4.2), one component k:
 *       sum_i |u_k(t1) - u_k(t0)| / sum_i |u_k(t1)|   (later level)
 *   LBM_RESIDUAL_CAVITY   Eq. cavity_creterion (Sec. 4.3), all components:
 *       sum_i sum_k |u_k(t1) - u_k(t0)| / sum_i sum_k |u_k(t1)|
 * The paper's intervals t1 - t0 (one step, one period T, 1000 steps) are
 * the caller's choice of reduction cadence.  A zero denominator gives 0 if
 * the numerator is 0, else +infinity.  component (0 = x, 1 = y, 2 = z) is
 * ignored by LBM_RESIDUAL_CAVITY.
 * Errors: EINVAL (null pointer, unknown kind, component outside 0..2, or
 * statistics without an earlier snapshot: prev_step < 0). */
enum lbm_residual_kind {
  LBM_RESIDUAL_STEADY = 0,
  LBM_RESIDUAL_PERIODIC = 1,
  LBM_RESIDUAL_CAVITY = 2
};
int lbm_stats_residual(const lbm_stats *s, int32_t kind, int32_t component, double *r);

/* The criterion `kind` of the handle's most recent reduction (as
 * lbm_read_stats, then lbm_stats_residual).  Synchronises.  EINVAL also if
 * no reduction has run since the last init, write or set_step. */
int lbm_residual(lbm_handle *h, int32_t kind, int32_t component, double *r);

/* Launch shape of the step kernel.  Affects speed, and (cells_per_thread
 * only) the FP32 rounding pattern: bx and by never change results; the two
 * cells of a pair are collided in packed FP32x2, where the compiler fuses
 * multiply-adds differently than in the one-cell kernel, so results agree to
 * FP32 rounding, not bit for bit. */
typedef struct lbm_launch {
  int32_t bx, by;           /* threads along x (multiple of 32, so a warp never
                               spans two x-rows) and y; bx*by <= 256          */
  int32_t cells_per_thread; /* 1, or 2: on even steps with nx even, each
                               thread updates the x-adjacent cells 2t, 2t+1,
                               moving each population of the pair as one
                               word (a warp touches 128 B per population
                               with 2-byte storage instead of 64 B); odd
                               steps run one cell per thread.  Stochastic
                               rounding draws the same random bits for a
                               cell either way.  Not for FP64 storage.
                               Q = 26 accepts 2 and runs one cell per
                               thread on every step.                        */
} lbm_launch;

/* Set / read the launch shape.  EINVAL if out of range. */
int lbm_set_launch(lbm_handle *h, const lbm_launch *launch);
int lbm_get_launch(lbm_handle *h, lbm_launch *launch);

/* Overlap of consecutive step launches (no counterpart in the paper; speed
 * only, results unchanged).  enable != 0 (the default): each step kernel is
 * launched as a programmatic dependent of the previous one, so its CTAs are
 * scheduled while the previous step drains and wait on the device for that
 * step's completion before reading any population.  0: plain stream order. */
int lbm_set_overlap(lbm_handle *h, int32_t enable);

/* Autotuner: time the step kernel on this domain for each candidate launch
 * shape (block shape, cells per thread; `trials` steps each, CUDA events on
 * the handle's stream) and keep the fastest.  The populations and step
 * counter are saved before and restored after, so the state is unaffected
 * (the chosen cells per thread sets the FP32 rounding pattern, see
 * lbm_set_launch); the choice is cached per (Q, storage, rounding, nx, ny,
 * nz) for later handles of the same shape.  trials <= 0
 * uses the cache only (or 8 trials on a miss).  Outputs may be NULL.
 * Synchronises; needs Q*N storage values of temporary device memory. */
int lbm_autotune(lbm_handle *h, int32_t trials, lbm_launch *chosen, double *ms_per_step);

/* ---- allocation-free reductions ------------------------------------------ */

/* The FP64 reductions of lbm_reductions for callers that cannot call
 * cudaMalloc.  The paper has no counterpart; this is a deployment aid.
 * Such callers include code whose device memory belongs to another
 * allocator with a fixed budget, latency-critical loops that must not pay
 * for cudaMalloc/cudaFree (cudaFree synchronises the whole device), and host
 * code running where CUDA allocation calls are not allowed.  Nothing is
 * allocated: the caller passes every input and output, and the only scratch
 * (one FP64 partial per thread block plus the final statistics, 983,160
 * bytes) is a static device array that each GPU loading the library keeps
 * until the process exits.
 *   desc, geom, params: the domain, as for lbm_create / set_geometry /
 *       set_params (host structs; rates are not used).
 *   step: the step counter n the populations belong to (its parity selects
 *       the storage layout; F(t_n) enters u).
 *   populations: device buffer of Q*N values of desc->storage in the
 *       library's storage layout at step n (for even n: canonical
 *       populations, [a][cell]).
 *   u_prev: device buffer of 3*N doubles, or NULL.  If non-NULL it receives
 *       the current velocity (the next call's snapshot), and if also
 *       prev_step >= 0 the residual sums compare against its old contents,
 *       which the caller states were taken at prev_step.
 *   out: host struct, filled as by lbm_reductions.
 *   cuda_stream: cudaStream_t the work runs on (NULL = legacy stream);
 *       the call synchronises it.
 * Limits: N = nx*ny*nz <= 2,097,152 cells (128^3); larger domains are
 * rejected with LBM_EINVAL and a message naming the limit.
 * The first call on a device looks up the static array's device address
 * (cudaGetSymbolAddress) with that device current.  The looked-up address
 * is kept for the life of the process: after a cudaDeviceReset of that
 * device it is stale, so the entry point must not be called on a device
 * that has been reset.  Every call on a device shares the same static
 * array: each call overwrites everything it reads, so nothing needs
 * clearing, but calls whose GPU work overlaps (e.g. on two streams at once)
 * race on it and must be serialised by the caller.
 * Errors: EINVAL (null pointer, bad sizes, kinds or storage; N too large),
 * ECUDA. */
int lbm_reductions_static(const lbm_desc *desc, const lbm_geom *geom,
                          const lbm_params *params, int64_t step, const void *populations,
                          double *u_prev, int64_t prev_step, lbm_stats *out,
                          void *cuda_stream);

/* Device memory the handle holds, in bytes. */
int lbm_memory_bytes(lbm_handle *h, int64_t *bytes);

/* The handle's population buffer: *ptr receives its device address and
 * *bytes its size (Q*N storage values).  The values are in the storage layout
 * of the current step counter's parity (for an even step the canonical
 * populations [a][cell]; for an odd step the post-collision values of the
 * previous step in the slots the in-place streaming keeps them in), so the
 * buffer can be handed to lbm_reductions_static with lbm_get_step's counter.
 * The handle keeps ownership; the address stays valid until lbm_destroy.
 * Reading it races with queued steps unless the caller orders the read after
 * them on the handle's stream; writing it is the caller's responsibility.
 * No synchronisation. */
int lbm_device_populations(lbm_handle *h, void **ptr, int64_t *bytes);

/* ---- batches of independent domains -------------------------------------- */

/* A batch advances many independent domains (different sizes, Q, storage,
 * step counters; Q = 14 or 18) together.  Grouped mode (default): each step
 * is one launch per group of domains sharing Q, storage, rounding and parity.  Persistent
 * mode: one cooperative launch runs a whole chunk of steps of all domains,
 * with a bounded grid barrier between steps.  The launches of a chunk are
 * captured once in a CUDA graph and replayed.  Each domain computes exactly
 * what a single-domain handle with one cell per thread computes, so a
 * domain's result is the same alone and in any mix.  Batched domains store
 * FP32, FP16 or BF16. */
typedef struct lbm_batch lbm_batch;

/* Up to `capacity` domains whose population buffers together stay within
 * `budget_bytes` (<= 0: no limit).  Work is queued on `cuda_stream`. */
int lbm_batch_create(int32_t capacity, int64_t budget_bytes, void *cuda_stream,
                     lbm_batch **out);
void lbm_batch_destroy(lbm_batch *b);

/* Add a domain (stream-ordered allocation of Q*N storage values, f = 0,
 * step 0); returns its slot.  EBUSY if no slot is free or the budget would
 * be exceeded; EINVAL for bad descriptors (as lbm_create/set_geometry/
 * set_params) and for LBM_NEQ_* faces (single-domain handles only). */
int lbm_batch_add(lbm_batch *b, const lbm_desc *desc, const lbm_geom *geom,
                  const lbm_params *params, int32_t *slot);

/* Remove a domain; its slot and memory are reused (stream-ordered free). */
int lbm_batch_remove(lbm_batch *b, int32_t slot);

/* As lbm_init_equilibrium for one domain (device arrays or NULL only). */
int lbm_batch_init_equilibrium(lbm_batch *b, int32_t slot, const double *u, const double *p,
                               int on_device);

/* Advance every active domain by nsteps, `chunk` steps per launch (or per
 * graph replay).  Asynchronous.  Returns LBM_ETIMEOUT if a grid barrier of
 * an earlier launch timed out. */
int lbm_batch_step(lbm_batch *b, int64_t nsteps, int32_t chunk);

int lbm_batch_get_step(lbm_batch *b, int32_t slot, int64_t *n);

/* As lbm_read_fields for one domain, into a device buffer.  Synchronises. */
int lbm_batch_read_fields(lbm_batch *b, int32_t slot, unsigned mask, void *dst,
                          int dst_on_device, int dtype);

/* As lbm_reductions for one domain (snapshot kept per domain). */
int lbm_batch_reductions(lbm_batch *b, int32_t slot, lbm_stats *out);

/* Reductions of every active domain, queued together with one
 * synchronisation: out[k] belongs to slots[k], k < *count.  Both arrays
 * must hold `capacity` entries. */
int lbm_batch_reductions_all(lbm_batch *b, lbm_stats *out, int32_t *slots, int32_t *count);

/* The criterion `kind` (see lbm_stats_residual) of the slot's most recent
 * reduction (lbm_batch_reductions or lbm_batch_reductions_all).  Host only,
 * no synchronisation.  EINVAL also if the slot has had no reduction since it
 * was added or initialised. */
int lbm_batch_residual(lbm_batch *b, int32_t slot, int32_t kind, int32_t component, double *r);

/* Launch shape of the batch kernels (bx multiple of 32, bx*by <= 256) and
 * mode: grouped (0: one launch per domain group per step) or persistent (1:
 * one cooperative launch per chunk, grid barrier between steps; a batch
 * holding a stochastically rounded domain runs grouped).  Speed only. */
int lbm_batch_set_launch(lbm_batch *b, int32_t bx, int32_t by, int32_t persistent);

/* Work split and order of grouped mode (no counterpart in the paper; speed
 * only, results are unchanged).
 *   tiles_per_cta: consecutive tiles (one tile = bx x by cells of one
 *     z-plane) each CTA of a group launch updates; 0 picks it from the
 *     group size.
 *   solo_min_cells: a domain with at least this many cells runs as its own
 *     launch of the single-domain update every step instead of sharing a
 *     group launch; 0 = two waves of resident CTAs, < 0 = never.  A domain
 *     with no partner in its group also runs solo.
 *   cluster_bytes: the active domains are packed into L2 clusters of at most
 *     this many population bytes (a larger domain forms its own); the steps
 *     of a chunk run in blocks of up to 32, and within a block each cluster
 *     runs all the block's steps before the next cluster starts, so its
 *     populations stay in L2 between steps.  0 = half of the device's
 *     L2, < 0 = one cluster (every domain advances step by step
 *     together).
 * Synchronises the batch's stream; the next step regroups.  Returns
 * LBM_EINVAL for tiles_per_cta outside 0..4096. */
int lbm_batch_set_schedule(lbm_batch *b, int32_t tiles_per_cta, int64_t solo_min_cells,
                           int64_t cluster_bytes);

/* Active domains, bytes of population storage, total cells. */
int lbm_batch_info(lbm_batch *b, int32_t *active, int64_t *used_bytes, int64_t *total_cells);

/* Test hook for the time-out path of the persistent grid barrier: the
 * barrier waits for `extra_arrivals` CTAs beyond the grid (that never come)
 * and gives up after `spin_limit` polls, so the next lbm_batch_step reports
 * LBM_ETIMEOUT.  (0, 1 << 26) restores normal operation. */
int lbm_batch_set_barrier_test(lbm_batch *b, int32_t extra_arrivals, int64_t spin_limit);

/* Message for the calling thread's most recent failure ("" if none). */
const char *lbm_last_error(void);
const char *lbm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
