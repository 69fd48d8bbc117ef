/*
 * aleweno.h -- C ABI of the GB300 (sm_103a) library for the cell-centred
 * ALE ADER-WENO finite volume scheme with time-accurate local time stepping
 * (LTS) on moving unstructured triangles (Boscheri, Dumbser, Zanotti).
 *
 * One context = one mesh (or one batch of independent meshes) resident on
 * one GPU.  The library owns every device allocation of a context.  All
 * arithmetic of the scheme runs in the library's CUDA kernels in FP64.
 *
 * Pointers: every array argument may be a host pointer or a device pointer
 * (CUDA unified addressing decides); arrays are row-major, the last index
 * fastest.  Layouts:
 *   Q, QM   [n_tris][4]  conserved variables (rho, rho u, rho v, rho E)
 *   HM      [n_tris][3]  geometric memory variable (x, y, t components)
 *   t, dt   [n_tris]     element time and time step in integer ticks;
 *                        1 tick = t_end / 2^time_quantum_log2
 *   X       [n_tris][6]  the element's own vertex coordinates x0,y0,x1,y1,x2,y2
 *   qhat    [n_tris][N_st][4] predictor degrees of freedom at the space-time
 *                        nodes l = tau_index * Mc + s, where s runs over the
 *                        degree-M lattice (i/M, j/M), j outer, i inner, and
 *                        tau_index over the M+1 Gauss-Lobatto times in [0,1];
 *                        Mc = (M+1)(M+2)/2, N_st = Mc (M+1)
 *   node X  [n_nodes][2], node t [n_nodes] ticks
 *
 * Errors: every entry point returns AW_OK (0) or a negative AW_ERR_* code and
 * leaves a message for aw_last_error().  No exception crosses the ABI.  Calls
 * on one context are not thread-safe; different contexts are independent.
 *
 * Devices: a context lives on the device that is current when aw_create is
 * called (its stream, memory and captured graphs belong to it).  Every entry
 * point taking a context makes that device current for the call and gives the
 * caller's current device back before returning.
 */
#ifndef ALEWENO_H
#define ALEWENO_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  AW_OK = 0,
  AW_ERR_INVALID_ARG = -1, /* bad argument or unsupported option */
  AW_ERR_BAD_MESH = -2,    /* clockwise or non-manifold element, too few elements for a stencil */
  AW_ERR_NONPHYSICAL = -3, /* rho <= 0, p <= 0 or an inverted element after an update */
  AW_ERR_DEADLOCK = -4,    /* no element satisfies the update criterion although some are unfinished */
  AW_ERR_TIMEOUT = -5,     /* a bounded device wait ran out */
  AW_ERR_CUDA = -6,        /* a CUDA runtime call failed */
  AW_ERR_STATE = -7        /* called before a mesh/state was loaded, or after a failed sweep */
};

typedef struct aw_ctx aw_ctx;

typedef struct {
  int order_M;            /* polynomial degree M in {1, 2, 3}: order M+1 in space and time */
  double gamma;           /* ratio of specific heats of the ideal gas, eq. eos */
  double cfl;             /* CFL number of the local time step, eq. timestep (<= 0.5) */
  int time_quantum_log2;  /* K in [1, 50]: t_end is 2^K ticks */
  double t_end;           /* final time t_f */
  int gts;                /* 0: local time stepping; 1: global step = min of local steps */
  int predictor_iters;    /* Picard iterations of eq. CGfinal; <= 0 selects M+1 */
  int mesh_velocity;      /* 0: V = v, the fluid velocity (Sec. 3); 1: V = 0 (Eulerian) */
  void* cuda_stream;      /* cudaStream_t to run on, or NULL for a stream the context creates */
  int flux;               /* 0: Rusanov-type ALE flux (eq. rusanov); 1: Osher-type ALE flux (eq. osher)
                             on the straight path (eq. path), path integral by 3-point Gauss-Legendre */
  double wall_u, wall_v;  /* velocity of the moving slip walls (boundary tag 2), the piston of Sec. 3.5:
                             their nodes move with it, the outer state mirrors the momentum normal to
                             the wall relative to it, and an element with such an edge counts the wall's
                             speed in its local step */
  double t_switch;        /* > 0: until t_switch every element takes the global minimum of the local
                             steps computed with CFL cfl_start, clipped at t_switch; local steps after
                             (the start of the Saltzman run, Sec. 3.5); 0: none */
  double cfl_start;
  double kidder[5];       /* r_i0, r_e0, rho_i0, rho_e0, s0 of the isentropic compression of Sec. 3.4
                             (eqs. KidderIC, KidderEx): edges tagged 3 take its exact state at each
                             quadrature point's position and time as outer state */
} aw_config;

/* Create a context (Sec. 2.1 set-up).  INVALID_ARG on an unsupported config. */
int aw_create(const aw_config* cfg, aw_ctx** out);
void aw_destroy(aw_ctx* ctx);
const char* aw_last_error(const aw_ctx* ctx);

/* Load a conforming triangulation (Sec. 2.1, eq. trian) and run the
 * pre-processing of Sec. 2.2: edges, Voronoi neighbourhoods, the seven
 * reconstruction stencils per element and the symmetric total stencil S^W
 * (eq. WENOstencil).  tri: [n_tris][3] counter-clockwise node indices;
 * bc: [n_tris][3] tag of local edge e = (v_e, v_{e+1 mod 3}): -1 interior,
 * 0 slip wall, 1 transmissive, 2 slip wall moving with (wall_u, wall_v),
 * 3 the exact state of the Kidder compression (cfg.kidder); shift: [n_tris][3][2] int8 periodic image of
 * each corner (corner = xy[node] + shift * period) or NULL, with period [2]
 * or NULL (both or neither); a zero period component means the mesh is not
 * periodic in that direction (the shock tubes of Sec. 3.2 are periodic in y
 * only), a negative one or two zeros are INVALID_ARG.  The arrays are copied.
 * BAD_MESH on invalid input. */
int aw_load_mesh(aw_ctx* ctx, int64_t n_nodes, const double* xy, int64_t n_tris,
                 const int32_t* tri, const int8_t* bc, const int8_t* shift,
                 const double* period);

/* Load n_inst independent, non-periodic meshes as one batch: every sweep then
 * advances all instances together (their stencils never meet, so each
 * instance evolves exactly as it would alone).  Instance k owns nodes
 * [node_offsets[k], node_offsets[k+1]) and triangles [tri_offsets[k],
 * tri_offsets[k+1]) of the concatenated xy [n_nodes][2], tri [n_tris][3] and
 * bc [n_tris][3]; tri holds node indices local to the instance; offsets start
 * at 0 (n_inst + 1 entries each).  t_end [n_inst] is the final time of each
 * instance; its tick is t_end[k] / 2^time_quantum_log2 (cfg.t_end is not
 * used).  aw_load_state then takes the concatenated averages.  Errors as
 * aw_load_mesh. */
int aw_load_batch(aw_ctx* ctx, int n_inst, const int64_t* node_offsets, const int64_t* tri_offsets,
                  const double* t_end, const double* xy, const int32_t* tri, const int8_t* bc);

/* Pre-processing phase of Sec. 2.6: cell averages Q [n_tris][4] at t = 0,
 * first WENO reconstruction, local time steps (eq. timestep), predictor;
 * all node and element times set to 0.  NONPHYSICAL if rho or p <= 0. */
int aw_load_state(aw_ctx* ctx, const double* Q);

/* aw_load_state on node positions xy [n_nodes][2] (host or device pointer)
 * instead of the mesh's own: element corners become xy[tri] plus their
 * periodic offsets.  The mesh pre-processing of aw_load_mesh (stencils,
 * total stencils, wall normals) is kept, so a small move of the nodes changes
 * the result smoothly.  BAD_MESH if an element turns clockwise. */
int aw_load_state_xy(aw_ctx* ctx, const double* Q, const double* xy);

/* One cycle of the LTS algorithm (Sec. 2.6): every element satisfying the
 * update criterion on S^W (eq. WENOupdate) moves its nodes (Sec. 2.4),
 * computes the space-time edge and vertex fluxes (eqs. spacetimenodes,
 * rusanov, STint), updates its average with the memory variable (eqs.
 * PDEfinal, Qm2), re-reconstructs on the virtual stencil (eqs. virtGeom,
 * virtCellaverage, weno), takes a new local step and runs its predictor.
 * *n_updated = number of elements updated (0 once all reached t_end).
 * DEADLOCK, NONPHYSICAL or CUDA on failure. */
int aw_lts_sweep(aw_ctx* ctx, int64_t* n_updated);

/* One global time step (the GTS reference of Sec. 3.2): requires gts = 1. */
int aw_gts_step(aw_ctx* ctx, int64_t* n_updated);

/* Run sweeps until every element reached the sync time min(t, t_end), or
 * max_sweeps sweeps ran (the computational phase of Sec. 2.6 runs every element
 * to a time).  A sync time before t_end follows the same rule as the final
 * time: every local step is clipped so that it ends at or before the sync
 * time, and elements stop there; the run to t is then the run whose final
 * time is t.  Moving the sync time back (below steps already taken) cuts
 * each step that crosses it and re-solves that element's predictor over the
 * shorter step from its own tau = 0 dofs; moving it forward gives each
 * element stopped at the old sync time its reconstruction, local step and
 * predictor there.  The sync time stays until the next aw_advance_to
 * (aw_lts_sweep updates nothing once every element reached it);
 * aw_load_state resets it to t_end.  t < t_end must be a whole number of
 * ticks and not behind any element's time; INVALID_ARG otherwise, for a
 * batch, or with a frozen schedule (aw_schedule mode 1 or 2).  Outputs may be
 * NULL: *sweeps_done counts sweeps that updated at least one element. */
int aw_advance_to(aw_ctx* ctx, double t, int64_t max_sweeps, int64_t* sweeps_done,
                  int64_t* updates_done);

/* Enqueue n sweeps on the context's stream without waiting (device-resident
 * benchmark loop); a later aw_sync() reports errors and the update count. */
int aw_enqueue_sweeps(aw_ctx* ctx, int64_t n);
int aw_sync(aw_ctx* ctx, int64_t* updates_since_last_sync);

/* State access (any argument may be NULL to skip it). */
int aw_get_state(aw_ctx* ctx, double* Q, double* t_elem);
int aw_get_nodes(aw_ctx* ctx, double* xy, double* t_node);
int aw_get_update_counts(aw_ctx* ctx, int64_t* per_elem, int64_t* total);
int aw_get_elem_arrays(aw_ctx* ctx, double* Q, double* QM, double* HM, int64_t* t,
                       int64_t* dt, double* X, int64_t* count, double* qhat);
/* Replace the whole LTS state (checkpoint restore / parity snapshots); all
 * element arrays and both node arrays are required. */
int aw_set_elem_arrays(aw_ctx* ctx, const double* Q, const double* QM, const double* HM,
                       const int64_t* t, const int64_t* dt, const double* X,
                       const int64_t* count, const double* qhat);
int aw_get_node_arrays(aw_ctx* ctx, double* X, int64_t* t);
int aw_set_node_arrays(aw_ctx* ctx, const double* X, const int64_t* t);

/* out[0] = largest GCL residual |sum of int n dS| / |T| seen in an update
 * (eq. gcl); out[1] = number of element updates; out[2] = sweeps run;
 * out[3] = space-time edge surfaces integrated (Sec. 2.5, eq. spacetimenodes).
 * out holds 4 doubles. */
int aw_diagnostics(aw_ctx* ctx, double* out);
/* Sizes (out has 6 entries): out[0] n_tris, out[1] n_nodes, out[2] n_edges,
 * out[3] N_st, out[4] total S^W entries, out[5] total distinct members of
 * the seven reconstruction stencils (without the element itself). */
int aw_sizes(aw_ctx* ctx, int64_t* out);

/* Per-kernel timing of sweeps with CUDA events recorded on the context's
 * stream between the launches (a second captured graph with an event record
 * between the kernels; each profiled sweep waits for its last event).  aw_profile_enable(ctx, 1) resets and starts
 * it; aw_profile_read fills ms[k] (total milliseconds of kernel k over the
 * profiled sweeps, k < the return value) and *sweeps, and returns the number
 * of kernels per sweep; aw_kernel_name(k) names kernel k (NULL if out of
 * range).  Recording adds a few microseconds per sweep. */
int aw_profile_enable(aw_ctx* ctx, int on);
int aw_profile_read(aw_ctx* ctx, double* ms, int64_t* sweeps);
const char* aw_kernel_name(int k);

/* The set of elements that satisfy the update criterion in the context's
 * current state (the elements the next aw_lts_sweep will update), computed
 * without allocating any memory.  No counterpart in the paper: it exists for
 * callers that cannot call cudaMalloc -- code running between the launches of
 * an application that owns all device memory through its own pool, or a
 * latency-critical loop where cudaMalloc's implicit device synchronisation is
 * not acceptable.  The work runs on the context's device (current at
 * aw_create), whichever device is current at the call; the caller's device is
 * given back.  The caller passes the outputs: ready_out, a device array
 * with room for n_tris int32, receives the ready element indices in ascending
 * order; n_ready_out, a device int64, receives their number.  The work is
 * enqueued on the context's stream and not waited for.  Scratch is a fixed
 * 16 KB array in device memory that every GPU loading the library holds until
 * the process exits; the first call for a device looks that device's copy up
 * (cudaGetSymbolAddress, with the context's device current), so make that
 * first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (other streams,
 * other contexts) race and must be serialised by the caller.  Meshes with more
 * than 1,048,576 triangles are rejected with AW_ERR_INVALID_ARG; STATE without
 * a loaded state. */
int aw_ready_set_noalloc(aw_ctx* ctx, int32_t* ready_out, int64_t* n_ready_out);

/* Frozen schedule.  The local time steps are integers of ticks taken from
 * the CFL bound (eq. timestep) through floor(), so the solution is a
 * piecewise-smooth function of the data with jumps wherever a step changes
 * by one tick.  mode 1 (record) logs the step every element takes at each of
 * its first k updates (update 0 is the step of aw_load_state) into a log
 * owned by the context; mode 2 (replay) takes the logged steps instead of
 * the CFL steps, so runs from perturbed data follow the recorded schedule
 * and differ smoothly; mode 0 returns to CFL steps.  The log survives
 * aw_load_state and is dropped with the mesh.  Local time stepping only
 * (INVALID_ARG with gts = 1).  An update beyond k stops the run with STATE.
 * aw_get_schedule copies the log, [n_tris][k] int64 ticks, to out (host or
 * device).  Changing the mode re-captures the sweep graph. */
int aw_schedule(aw_ctx* ctx, int mode, int64_t k);
int aw_get_schedule(aw_ctx* ctx, int64_t* out);

/* Adjoint of n LTS sweeps for the schedule they take (the sweep map with the
 * ready sets and tick steps held fixed, and the mesh pre-processing of
 * aw_load_mesh held fixed).
 * aw_adjoint_forward runs n_sweeps sweeps from a state just loaded by
 * aw_load_state / aw_load_state_xy and keeps a device checkpoint of the
 * state every ckpt_every sweeps (plus the final state); STATE if a sweep ran
 * since the load.  aw_adjoint then takes dJ/d(final state) of a scalar J --
 * dJdQ [n_tris][4] conserved averages, dJdX [n_tris][6] element corners,
 * dJdxy [n_nodes][2] node positions, each NULL for zero, host or device
 * pointers -- and writes dJ/dQ0 [n_tris][4] and dJ/dxy0 [n_nodes][2] with
 * respect to the loaded averages and node positions (either may be NULL).
 * It recomputes each segment of ckpt_every sweeps from its checkpoint and
 * reverses the sweeps of the segment one by one: phase B of the ready
 * elements (predictor iterations, characteristic WENO weights and
 * least-squares solves, virtual projection), then the node commit, the FV
 * update and memory variables, the edge fluxes and the node solver.  Device
 * memory: (n_sweeps / ckpt_every + ckpt_every + 3) copies of the state.  The
 * context is left in the final state; aw_adjoint may be called again for
 * another J.  STATE if a positivity safeguard (scaling of w_h, predictor
 * fallback) acted in one of the sweeps: the map has a kink there.  The
 * adjoint covers the Rusanov-type flux (flux = 0); INVALID_ARG otherwise.
 * No counterpart in the paper. */
int aw_adjoint_forward(aw_ctx* ctx, int64_t n_sweeps, int64_t ckpt_every);
int aw_adjoint(aw_ctx* ctx, const double* dJdQ, const double* dJdX, const double* dJdxy,
               double* dJdQ0, double* dJdxy0);

/* Tile shapes of the sweep kernels; they change no result, only speed.
 * tiles[0] = 1 halves the reconstruction's elements per block (16/8/4 for
 * P1/P2/P3 by default on 256 threads; half of them on 128 threads),
 * tiles[1] = 1 runs the predictor on 256-thread blocks (default 128), tiles[2] = blocks per SM of the kernels that loop over a
 * sweep's lists (default 8, range 1..64).  Setting them re-captures the sweep
 * graph.  No counterpart in the paper. */
int aw_set_tiles(aw_ctx* ctx, const int32_t* tiles);
int aw_get_tiles(aw_ctx* ctx, int32_t* tiles);

/* Autotuner of the tile shapes on the loaded state: each of 12 candidates
 * (tiles[0] in {0,1} x tiles[1] in {0,1} x tiles[2] in {4,8,16}; candidate k
 * = tiles[0]*6 + tiles[1]*3 + index of tiles[2]) runs the same n_sweeps
 * sweeps from the current state twice, timed with CUDA events on the
 * context's stream; ms[k] (NULL to skip) receives the faster of the two
 * times and best[3] the fastest shape, which the context keeps.  The state is restored afterwards.  Needs
 * one extra copy of the state in device memory.  No counterpart in the
 * paper. */
int aw_autotune(aw_ctx* ctx, int64_t n_sweeps, double* ms, int32_t* best);

/* Host-only check of the adjoint's element-level pieces (no GPU needed): for
 * order M and a seed, each reverse (reconstruction, predictor, edge flux,
 * node solver) is compared with central differences of its forward on
 * random smooth data; report[0..3] receive the largest relative mismatches.
 * No counterpart in the paper. */
int aw_adjoint_selftest(int order_M, uint64_t seed, double* report);

/* Measured FP64 FMA throughput of the current GPU (GFLOP/s), a roofline
 * denominator: a fixed dependent-chain DFMA kernel over all SMs. */
int aw_measure_fp64_peak(double* gflops);

#ifdef __cplusplus
}
#endif
#endif
