/*
 * CPU oracle of the cell-centred ALE ADER-WENO finite volume scheme with
 * time-accurate local time stepping (Boscheri, Dumbser, Zanotti).
 *
 * TEST INFRASTRUCTURE ONLY.  This plain, serial FP64 C implementation exists
 * to check the CUDA path; only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or helper with the CUDA library.
 *
 * Array layouts match the C ABI of the CUDA library (row-major, the last
 * index fastest):
 *   Q, QM      [n_tris][4]   conserved (rho, rho u, rho v, rho E)
 *   HM         [n_tris][3]   geometric memory (x, y, t components)
 *   t, dt      [n_tris]      int64 ticks, 1 tick = t_end / 2^K
 *   X          [n_tris][6]   own vertex coordinates x0,y0,x1,y1,x2,y2
 *   qhat       [n_tris][N_st][4], space-time node l = tau_index*Mc + s
 *   node X     [n_nodes][2], node t [n_nodes] int64 ticks
 */
#ifndef AW_ORACLE_H
#define AW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oc_ctx oc_ctx;

typedef struct {
  int order_M;          /* polynomial degree M in {1,2,3} */
  double gamma;         /* ratio of specific heats */
  double cfl;           /* CFL number, eq. timestep */
  int time_quantum_log2;/* K: t_end is 2^K ticks */
  double t_end;
  int gts;              /* 1: global time step (min of local steps) */
  int predictor_iters;  /* Picard iterations of eq. CGfinal; <=0 means M+1 */
  int mesh_velocity;    /* 0: V = v (Lagrangian-type), 1: V = 0 (Eulerian) */
  int flux;             /* 0: Rusanov-type (eq. rusanov), 1: Osher-type (eq. osher) */
  double wall_u, wall_v; /* velocity of the moving slip walls (bc 2), Sec. 3.5 piston */
  double t_switch;      /* > 0: global steps with CFL cfl_start until t_switch, then
                           local steps (the start of the Saltzman run, Sec. 3.5) */
  double cfl_start;
  double kidder[5];     /* r_i0, r_e0, rho_i0, rho_e0, s0: the exact isentropic
                           compression (Sec. 3.4) whose state bc-3 edges take */
} oc_config;

int oc_create(const oc_config* cfg, oc_ctx** out);
void oc_destroy(oc_ctx* c);
const char* oc_last_error(const oc_ctx* c);
int oc_load_mesh(oc_ctx* c, int64_t n_nodes, const double* xy, int64_t n_tris,
                 const int32_t* tri, const int8_t* bc, const int8_t* shift,
                 const double* period);
int oc_load_state(oc_ctx* c, const double* Q);
/* oc_load_state on node positions xy [n_nodes][2]; stencils, total stencils
   and wall normals stay those chosen by oc_load_mesh */
int oc_load_state_xy(oc_ctx* c, const double* Q, const double* xy);
/* frozen schedule (reading R12): mode 1 records the dt ticks every element
   takes at each of its first k updates (count 0 = the initial step), mode 2
   replays them instead of the CFL steps, mode 0 returns to free steps; the
   log survives oc_load_state so that perturbed runs replay a base run */
int oc_schedule(oc_ctx* c, int mode, int64_t k);
int oc_get_schedule(const oc_ctx* c, int64_t* out); /* [n_tris][k] */
/* load a schedule log [n_tris][k] (the layout oc_get_schedule returns);
   oc_schedule(c, 2, 0) then replays it */
int oc_set_schedule(oc_ctx* c, int64_t k, const int64_t* log);
int oc_sweep(oc_ctx* c, int64_t* n_updated);
/* sweeps until every element reached the sync time t (t_end, or a whole
   number of ticks not behind any element: reading R18) or max_sweeps ran */
int oc_advance_to(oc_ctx* c, double t, int64_t max_sweeps, int64_t* sweeps_done, int64_t* updates_done);
int oc_get_elem(const oc_ctx* c, double* Q, double* QM, double* HM, int64_t* t,
                int64_t* dt, double* X, int64_t* count, double* qhat);
int oc_set_elem(oc_ctx* c, const double* Q, const double* QM, const double* HM,
                const int64_t* t, const int64_t* dt, const double* X,
                const int64_t* count, const double* qhat);
int oc_get_nodes(const oc_ctx* c, double* X, int64_t* t);
int oc_set_nodes(oc_ctx* c, const double* X, const int64_t* t);
int64_t oc_n_st(const oc_ctx* c);
int64_t oc_n_edges(const oc_ctx* c);
/* diagnostics: [0] max GCL residual / |T|, [1] number of updates checked */
int oc_diag(const oc_ctx* c, double* out);
/* stencils of element i: members[7][n_e] (-1 where a stencil was dropped),
   total stencil S^W (returns its size; writes up to cap entries) */
int oc_get_stencils(const oc_ctx* c, int64_t i, int32_t* members, int32_t* sw, int cap);
/* Debug entry points used by the pin tests. */
int oc_reconstruct_eval(oc_ctx* c, int64_t i, int64_t npts, const double* xy, double* out);
int oc_predict_debug(oc_ctx* c, const double* X6, double dt_sec, const double* w_nodal,
                     double* qhat_out);
/* the configuration's numerical flux; qR NULL: boundary state of type bc built
   from qL (a wall mirrors the normal momentum, a moving wall the normal
   momentum relative to the wall; transmissive copies qL: in a sweep the
   transmissive outer state is the element average instead, R15) */
int oc_flux_debug(const oc_ctx* c, const double* qL, const double* qR, const double* n3,
                  int bc, double* out);
int oc_eval_qh(const oc_ctx* c, const double* qhat, int64_t npts, const double* pts, double* out);
/* tables: what = 0 Dubiner at points (npts x Mc), 1 Sigma (Mc x Mc),
   2 GLL nodes (M+1), 3 K_t ((M+1)^2), 4 M_t ((M+1)^2), 5 lattice nodes (Mc x 2),
   6 Gauss-Legendre nodes+weights on [0,1] for n=npts (2n),
   7 spatial Lagrange basis at points (npts x Mc) */
int oc_table(const oc_ctx* c, int what, int64_t npts, const double* pts, double* out);

#ifdef __cplusplus
}
#endif
#endif
