/*
 * ugmech.h -- C ABI of a GB300 (sm_103a) library for the mechanical-interaction
 * step of spherical cell agents, after Hesam et al., "GPU Acceleration of 3D
 * Agent-Based Biological Simulations" (arXiv 2105.00039).
 *
 * One step (Sec. III and Sec. IV-A of the paper):
 *   1. rebuild a uniform grid whose box edge is the largest agent diameter
 *      (Sec. IV-A, Fig. 4) and sort the agents by box (Sec. IV-D sorts agent
 *      state along a space-filling order so that neighbours share cache lines);
 *   2. for every agent, visit the 27 surrounding boxes and sum the pairwise
 *      sphere-sphere force of Eq. 1 over overlapping pairs;
 *   3. test adherence, integrate and cap the displacement (Sec. III, the
 *      paragraph after Eq. 1), and move the agent.
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers owned by the caller unless a
 *     comment says otherwise.  The library never allocates device memory;
 *     scratch space is a caller-provided workspace (`ws`, `ws_bytes`) whose
 *     size comes from the matching *_workspace_bytes function.  `ws` must be
 *     256-byte aligned.  Its contents need not be initialised and are
 *     clobbered.
 *   - Agent state is float32, 4 floats per agent: (x, y, z, diameter), 16-byte
 *     aligned.  Forces and gradients use the same 4-float rows.  At most 2^30
 *     agents per call (UG_EINVAL above).
 *   - max_boxes, the capacity of a box table, lies in [27, 2^31 - 256]
 *     (UG_EINVAL outside).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Every call is
 *     asynchronous: the return value reports argument and launch errors only.
 *     Errors found on the device (bad input values, grid too large, a list
 *     overflow) are written to `*status`, a device int32 the caller zeroes
 *     before the first call; the first error wins and later kernels of the
 *     same call become no-ops.  Read it after synchronising.
 *   - Calls on different streams must use different workspaces.  The library
 *     keeps no state between calls and is safe to call from several host
 *     threads with distinct workspaces.
 *   - n = 0 is valid and launches nothing.
 */
#ifndef UGMECH_H
#define UGMECH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define UG_OK               0
#define UG_EINVAL          (-1) /* bad argument: null pointer, bad size or alignment, nsteps < 0 */
#define UG_EBADSTATE       (-2) /* device: non-finite coordinate, or diameter not finite and > 0 */
#define UG_EGRID_TOO_LARGE (-3) /* device: the grid needs more than max_boxes boxes */
#define UG_ECAPACITY       (-4) /* device: a per-agent output list was too short */
#define UG_EWORKSPACE      (-5) /* ws_bytes smaller than the *_workspace_bytes figure */
#define UG_ETIMEOUT        (-6) /* reserved: no kernel of this library waits on another */
#define UG_ECUDA           (-7) /* a CUDA runtime call failed (launch, memset, copy) */

/* Human-readable text for a status code (static storage, never NULL). */
const char *ug_strerror(int status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int ug_version(void);

/* ------------------------------------------------------------------ types */

/* Mechanical constants.  k and gamma are Eq. 1's repulsion and attraction
 * coefficients.  The paper names the adherence test, the integration and the
 * displacement bound (Sec. III) without formulas; this library reads them as
 *   moving  <=>  |F| > adherence (strict)
 *   v = dt / m * F,  m = density * (pi/6) * diameter^3
 *   if |v| > max_disp: v *= max_disp / |v|   (max_disp = 0 freezes every agent,
 *                                              as in the paper's benchmark B)
 * contact_margin m_c widens every contact: delta = r1 + r2 + 2 m_c - |p1 - p2|
 * (R in Eq. 1 still uses the true radii), and the box edge grows by 2 m_c. */
typedef struct {
    float k;
    float gamma;
    float adherence;
    float dt;
    float density;
    float max_disp;
    float contact_margin;
} ug_params;

/* Geometry of one simulation's uniform grid (Sec. IV-A), written on the device.
 *   edge   = S + 8 ulp(C), S = largest diameter + 2 * contact_margin (the largest
 *            contact distance), C = max(S, largest |coordinate|); the 8 ulps keep
 *            every contact pair in adjacent boxes despite float32 rounding
 *   origin = (min corner of the agent centres) - edge, per axis
 *   box of an agent b = max(floor((p - origin) / edge), 1) per axis, in IEEE
 *   float32 round-to-nearest arithmetic; dims = box of the max corner + 2, so
 *   one empty layer of boxes surrounds the agents.
 *   Boxes are numbered row-major, x fastest: key = (bz*dims[1] + by)*dims[0] + bx,
 *   offset by box_base inside the table shared by all simulations of a call. */
typedef struct {
    float origin[3];
    float edge;
    int32_t dims[3];
    uint32_t box_base;   /* first box of this simulation in the shared table */
    uint32_t nboxes;     /* dims[0] * dims[1] * dims[2] (0 for an empty simulation) */
    uint32_t agent_base; /* first sorted slot of this simulation */
    uint32_t nagents;
    uint32_t reserved;
} ug_grid_info; /* 48 bytes */

/* Launch tuning for the batched step (autotuned by ug_tune_batched).
 *   agents_per_lane 2: each lane sweeps two box-sorted agents over their merged
 *                      neighbour runs (sweep_block is then fixed at 128);
 *                   1: one agent per lane with shared-memory staging, CTAs of
 *                      sweep_block threads.  0 = default (2).
 *   pair_mode       0: every agent sums its own pairs (as ug_step; default);
 *                   1: every pair evaluated once (as ug_step_pairs_once; the
 *                      two fields above are then ignored).  Either way a
 *                      simulation's result is bit-identical to the matching
 *                      single-simulation entry on its rows alone. */
typedef struct {
    int32_t sweep_block;      /* 64 or 128; 0 = default (128) */
    int32_t agents_per_lane;  /* 1 or 2; 0 = default (2) */
    int32_t pair_mode;        /* 0 or 1; 0 = default */
    int32_t neighbour_walk;   /* with pair_mode 1 (any number of simulations), or with
                                 agents_per_lane 2 and pair_mode 0 (one simulation):
                                 0 = each neighbour row cut to the x-window that can hold
                                 contacts where that pays, judged from n_total and
                                 max_boxes (n_total >= 2 max_boxes, about 6 neighbours
                                 per agent and up; every pair once: n_total >= 8
                                 max_boxes, about 24 and up), else the full three-box runs
                                 (default);
                                 1 = always the full runs; 2 = always the windows.  The
                                 same bits every way.  The other layouts walk full runs. */
    int32_t reserved[4];
} ug_tuning;

/* ------------------------------------------------------------------ workspace */

/* Bytes of workspace needed by ug_grid_build, ug_step, ug_step_pairs_once,
 * ug_step_traced and ug_step_batched for n agents in nsims simulations with
 * room for max_boxes grid boxes (summed over the simulations). */
size_t ug_workspace_bytes(uint32_t n, uint32_t nsims, uint32_t max_boxes);

/* ------------------------------------------------------------------ grid build */

/* Uniform-grid construction (Sec. IV-A, Fig. 4/5) with the agents reordered by
 * box (Sec. IV-D).  The paper keeps a per-box count and a linked list; here the
 * boxes are a counting sort: box_start[b] .. box_start[b+1] are the sorted slots
 * of box b, agents of one box keep their input order.
 *   state_in      [n] rows (x, y, z, d), any order
 *   perm_in       [n] id carried by each input row, or NULL for ids 0..n-1
 *   state_sorted  [n] out: rows in box order
 *   perm_sorted   [n] out: perm_sorted[s] = perm_in[input row placed at slot s]
 *   box_start     [max_boxes + 1] out: exclusive prefix of box counts; entries
 *                 0 .. info->nboxes are valid, box_start[nboxes] = n
 *   info          [1] out: the grid geometry
 * Device errors: UG_EBADSTATE (non-finite input or diameter <= 0),
 * UG_EGRID_TOO_LARGE (needs more than max_boxes boxes). */
int ug_grid_build(const float *state_in, const uint32_t *perm_in, uint32_t n,
                  float contact_margin, float *state_sorted, uint32_t *perm_sorted,
                  uint32_t *box_start, uint32_t max_boxes, ug_grid_info *info,
                  void *ws, size_t ws_bytes, int32_t *status, void *stream);

/* ug_grid_build for callers that cannot allocate device memory (the paper has
 * no counterpart: this is a library convenience).  Some callers are handed only
 * their inputs and outputs and may not allocate at the point of the call -- a
 * plug-in whose host application owns all of the GPU's memory, or code under a
 * fixed memory budget -- so they cannot supply ug_grid_build's workspace.  This
 * variant uses a fixed scratch array of about 14 MiB compiled into the library
 * (one per GPU that loads it, held until the process exits) and calls no
 * allocator.  Arguments and results are those of ug_grid_build, and its
 * argument checks come first (UG_EINVAL as there).
 *   Limits, checked after them: n <= 262144 and max_boxes <= 1048576, else
 *   UG_EWORKSPACE (the built-in scratch is too small) before any device work.
 *   The first call in a CUDA context looks up the array's address in that
 *   context (again after cudaDeviceReset, or in a context other than the
 *   device's primary one); make it before any stream capture.  Every call
 *   shares the array: calls that overlap on the GPU (other streams or host
 *   threads on the same device) race on it. */
int ug_grid_build_noalloc(const float *state_in, const uint32_t *perm_in, uint32_t n,
                          float contact_margin, float *state_sorted, uint32_t *perm_sorted,
                          uint32_t *box_start, uint32_t max_boxes, ug_grid_info *info,
                          int32_t *status, void *stream);

/* ------------------------------------------------------------------ forces */

/* Eq. 1 summed over every overlapping pair found in the 27 boxes around each
 * agent (Sec. IV-A).  Inputs are the outputs of ug_grid_build.
 *   force [n] out: (Fx, Fy, Fz, number of contacts) per sorted slot.
 * delta is evaluated in float-float arithmetic, so the contact predicate
 * delta > 0 and delta itself are exact to ~1e-12 of the contact distance; F is
 * accumulated with compensated (TwoSum) summation. */
int ug_compute_forces(const float *state_sorted, const uint32_t *box_start,
                      const ug_grid_info *info, uint32_t n, ug_params p, float *force,
                      int32_t *status, void *stream);

/* The contact pairs themselves (for checking the neighbour sets).
 *   count [n] out: contacts of each sorted slot
 *   nbr   [n * max_per_agent] out: sorted-slot indices of the contacts of slot s
 *         at nbr[s * max_per_agent + c], in visiting order
 * Device error UG_ECAPACITY if an agent has more than max_per_agent contacts
 * (count still holds the true number). */
int ug_list_pairs(const float *state_sorted, const uint32_t *box_start,
                  const ug_grid_info *info, uint32_t n, float contact_margin,
                  uint32_t max_per_agent, uint32_t *count, uint32_t *nbr,
                  int32_t *status, void *stream);

/* Adherence test, integration and displacement cap (Sec. III) for given forces.
 *   state_in  [n] rows; force [n] from ug_compute_forces
 *   state_out [n] out: moved rows (diameters copied); may alias state_in
 *   disp_out  [n] out, nullable: (ux, uy, uz, moving ? 1 : 0) */
int ug_apply_displacement(const float *state_in, const float *force, uint32_t n, ug_params p,
                          float *state_out, float *disp_out, int32_t *status, void *stream);

/* ------------------------------------------------------------------ fused steps */

/* nsteps full steps (grid rebuild + sweep + move each step), fused so that the
 * move, the next step's bounding box and the next grid's geometry are produced
 * by the sweep kernel.
 *   state [n] in/out: rows; on return in the box order of the last step
 *   perm  [n] in/out: id of each row (permuted along with the rows)
 * Deterministic: the same input gives bit-identical output. */
int ug_step(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
            uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream);

/* ug_step with every overlapping pair evaluated once (Newton's third law): each
 * agent walks only the forward half of its neighbourhood and the pair's force
 * is added to both agents as 64-bit fixed point (units of 2^-32, integer
 * atomics, so still deterministic), after which a second kernel moves the
 * agents.  Same arguments, workspace and results within the same tolerance as
 * ug_step, but not the same bits (fixed-point instead of compensated float32
 * sums).  It pays in dense grids: 1.2x at ~32 and 1.4x at ~64 neighbours per
 * agent on GB300 (from 8 agents per box of max_boxes its forward rows are cut
 * to the agents' x-windows, with the same bits), while on sparse grids (a few
 * agents per box) the atomics cost more than the halved walk saves and ug_step
 * is faster.  For many simulations use ug_step_batched with
 * tuning->pair_mode = 1. */
int ug_step_pairs_once(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
                       uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream);

/* ug_step with CUDA events recorded between its kernels, for per-kernel timing.
 *   events  HOST array of nevents cudaEvent_t handles created by the caller
 *   nevents >= 2 + 5 * nsteps.  events[0] precedes the bounding-box kernel;
 *           events[1 + 5t + k] precedes kernel k of step t (k = 0 key/histogram,
 *           1 scan, 2 placement, 3 stable in-box order, 4 sweep + move) and
 *           events[1 + 5(t+1)] follows step t's sweep. */
int ug_step_traced(float *state, uint32_t *perm, uint32_t n, ug_params p, int32_t nsteps,
                   uint32_t max_boxes, void *ws, size_t ws_bytes, int32_t *status, void *stream,
                   void *const *events, int32_t nevents);

/* Many independent simulations advanced together (each kernel of a step covers
 * all of them; there is one grid per simulation).  Simulation s owns rows
 * sim_offset[s] .. sim_offset[s+1]-1 of state and perm and never mixes with
 * the others; its result is bit-identical to ug_step (ug_step_pairs_once with
 * tuning->pair_mode 1) on its rows alone.
 *   sim_offset [nsims + 1] DEVICE, non-decreasing, sim_offset[nsims] = n_total
 *   params     [nsims] DEVICE, per-simulation constants
 *   max_boxes  capacity of the shared box table (sum over simulations)
 *   tuning     HOST pointer or NULL (defaults) */
int ug_step_batched(float *state, uint32_t *perm, const uint32_t *sim_offset, uint32_t nsims,
                    uint32_t n_total, const ug_params *params, int32_t nsteps,
                    uint32_t max_boxes, const ug_tuning *tuning, void *ws, size_t ws_bytes,
                    int32_t *status, void *stream);

/* Time each candidate configuration (one agent per lane with 64 or 128 threads
 * per CTA, two agents per lane, every pair once; the last two with the full
 * runs and with the windows, the two-agent windows for one simulation only) on
 * the given batched problem -- three fused
 * steps (grid build, sweep, move) of a scratch copy of the rows, after one
 * untimed step -- and write the fastest to *best (HOST pointer).  `state` is
 * only read.  Needs ws_bytes >= ug_workspace_bytes(n_total, nsims, max_boxes)
 * + 20 * n_total + 768.  Synchronises the stream. */
int ug_tune_batched(const float *state, const uint32_t *sim_offset, uint32_t nsims,
                    uint32_t n_total, const ug_params *params, uint32_t max_boxes,
                    ug_tuning *best, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------ adjoint */

/* Workspace for ug_step_backward over nsteps steps. */
size_t ug_backward_workspace_bytes(uint32_t n, uint32_t max_boxes, int32_t nsteps);

/* Reverse-mode derivative of nsteps steps (the adjoint of the step above; the
 * adherence test, the cap branch and contact membership are piecewise constant
 * and contribute no derivative).  The forward segment is recomputed from the
 * checkpoint, saving each step's grid, then swept in reverse.
 *   ckpt_state [n] rows at the start of the segment, in the row order ug_step
 *              was given (not modified)
 *   grad_out   [n] dL/d(rows after nsteps), in the row order ug_step returned
 *              (x, y, z, diameter components)
 *   grad_in    [n] out: dL/d(ckpt_state), in ckpt_state's row order
 *   grad_params[2] out (DEVICE): dL/dk, dL/dgamma contributed by this segment */
int ug_step_backward(const float *ckpt_state, uint32_t n, ug_params p, int32_t nsteps,
                     uint32_t max_boxes, const float *grad_out, float *grad_in,
                     float *grad_params, void *ws, size_t ws_bytes, int32_t *status,
                     void *stream);

/* ------------------------------------------------------------------ version ladder */

/* The paper's GPU versions (Sec. IV-B to IV-E), for comparison with the main
 * path only; it has no role in ug_step.  Forces of Eq. 1 on every agent of
 * `state`, evaluated directly (delta = r_i + r_j + 2 contact_margin - d, plain
 * sums) on the main path's grid geometry:
 *   version 0  one thread per agent over per-box linked lists (each box keeps
 *              its last agent, each agent the one added before it), rows in the
 *              caller's order, float64 arithmetic
 *   version 1  as 0 in float32
 *   version 2  as 1 over box-sorted rows (the main path's counting sort)
 *   version 3  one 32-thread CTA per box, the 27 boxes' agents appended to
 *              shared memory through an atomic counter, float32, box-sorted
 *              rows; a neighbourhood above 1024 agents records UG_ECAPACITY
 *   state      [n] DEVICE rows (x, y, z, diameter), caller's order, 16-B aligned
 *   force      [n][4] DEVICE float64 (fx, fy, fz, overlapping pairs), caller's
 *              order, 16-B aligned
 *   max_boxes  capacity of the grid (as for ug_grid_build)
 *   ws         >= ug_ladder_workspace_bytes(n, max_boxes), 256-B aligned
 * Versions 1-3 sum in an order set by atomics, so their float32 results may
 * differ in the last bits from run to run.  Errors: UG_EINVAL (version outside
 * 0..3, bad pointer or size), UG_EWORKSPACE, device errors as for ug_grid_build. */
size_t ug_ladder_workspace_bytes(uint32_t n, uint32_t max_boxes);
int ug_forces_ladder(int32_t version, const float *state, uint32_t n, ug_params p,
                     uint32_t max_boxes, double *force, void *ws, size_t ws_bytes, int32_t *status,
                     void *stream);

/* ------------------------------------------------------------------ symmetric pairs */

/* Symmetric (Newton's third law) evaluation of Eq. 1 (the force evaluation of
 * ug_step_pairs_once).  Same inputs and output layout as ug_compute_forces (rows,
 * box table and grid record of ug_grid_build; force[n] = (Fx, Fy, Fz,
 * overlapping pairs) per sorted row).  each_pair_once != 0: every agent walks
 * only the forward half of its neighbourhood (the plane above, the row above,
 * the rest of its own run), so each overlapping pair is evaluated once and its
 * force is added to both agents; 0: every agent walks all 27 boxes.  Sums are
 * accumulated as 64-bit fixed point (units of 2^-32) with integer atomics, so
 * both modes are deterministic and give the same bits; the float-float contact
 * test and Eq. 1 are the main path's, summed in fixed point rather than with
 * compensated float32 sums.  A pair force component of 2^30 or more records
 * UG_EBADSTATE; a per-agent sum holds |F| < 2^31 force units (with the
 * default constants and diameters ~10, Eq. 1's pair forces are a few tens of
 * units, far inside this range).
 *   ws  >= 32 * n bytes, 256-B aligned (the fixed-point accumulators) */
int ug_forces_symmetric(int32_t each_pair_once, const float *state_sorted, const uint32_t *box_start,
                        const ug_grid_info *info, uint32_t n, ug_params p, float *force, void *ws,
                        size_t ws_bytes, int32_t *status, void *stream);

/* ------------------------------------------------------------------ helpers */

/* perm[i] = i. */
int ug_iota(uint32_t *perm, uint32_t n, void *stream);

/* rows_by_id[perm[s]] = rows[s]  (undo the box order; perm must be a permutation). */
int ug_scatter_rows(const float *rows, const uint32_t *perm, uint32_t n, float *rows_by_id,
                    void *stream);

/* rows[s] = rows_by_id[perm[s]]  (apply the box order). */
int ug_gather_rows(const float *rows_by_id, const uint32_t *perm, uint32_t n, float *rows,
                   void *stream);

#ifdef __cplusplus
}
#endif

#endif /* UGMECH_H */
