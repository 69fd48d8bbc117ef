/*
 * CPU oracle of the cell-centred ALE ADER-WENO finite volume scheme with
 * time-accurate local time stepping on moving triangles (Boscheri, Dumbser,
 * Zanotti, "High order cell-centered Lagrangian-type finite volume schemes
 * with time-accurate local time stepping on unstructured triangular meshes").
 *
 * TEST INFRASTRUCTURE.  Plain, serial, FP64 and deliberately unoptimised:
 * every step follows the paper's text in its order and notation.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares nothing with the CUDA library.
 *
 * Readings of points the paper leaves open (the same readings bind the CUDA
 * library; each is restated where it is used):
 *  R1 times are int64 ticks, 1 tick = t_end/2^K; dt = floor(dt_cfl/tick),
 *     at least 1, clipped so that t + dt <= t_end (Sec. 2.1, eq. updateFV).
 *  R2 Jacobi sweep: the ready set and phase A (node motion, space-time fluxes,
 *     FV update) use the sweep-start state; phase B (projection, WENO, dt,
 *     predictor) runs on the post-update state (Sec. 2.6).  The paper fixes
 *     no order between ready neighbours, so the rule itself is parity
 *     unpinned; the sweep is pinned through what it must keep (GCL,
 *     conservation, free stream, LTS with equal steps = GTS, exact update
 *     counts, the exact Sod solution and the designed order).
 *  R3 stencil rule: central = n_e nearest centroids within M+1 vertex-
 *     neighbour layers; sector s = i plus the n_e-1 nearest elements whose
 *     centroid lies in the closed cone (primary: spanned by the rays from
 *     the centroid to the edge's vertices; reverse: the opposite cone)
 *     within M+2 layers, dropped when too few.  Distances at t=0, ties by
 *     element index.  S^W = union of stencils, edge neighbours and the
 *     vertices' Voronoi sets, closed under symmetry (Sec. 2.2).
 *  R4 constrained least squares: exact on T_i (w_0 = Q_i), least squares on
 *     the other members; Dubiner basis in T_i's reference frame; sigma sums
 *     1 <= alpha+beta <= M; the fields the weights act on are those of R10
 *     (eq. weno).
 *  R5 virtual geometry X~ = X^n + dt_j * int_0^tau* V_h(vertex) dtau and
 *     virtual average = reference-triangle average of q_h at tau*; a stencil
 *     element already at t_i uses its real data (eqs. virtGeom,
 *     virtCellaverage).
 *  R6 predictor nodes: equispaced degree-M lattice x (M+1) Gauss-Lobatto
 *     times; test functions of the tau>0 nodes; fixed M+1 Picard iterations;
 *     initial guess w_h at every time slice, geometry static (Sec. 2.3).
 *  R7 node velocity is the time average over [tau0,tau1], i.e. the node
 *     moves by sum_j mu_j dt_j int V_h dtau / sum_j mu_j (eqs. NodesVel,
 *     newVertex); wall nodes keep their tangential displacement, corners
 *     stay fixed.
 *  R8 one bilinear space-time surface per edge with a moved endpoint
 *     (a triangle is the same surface with one endpoint unmoved); each
 *     side's q_h at its reference edge point and its own tau; (M+1)^2 Gauss
 *     points (eqs. spacetimenodes, rusanov, STint).
 *  R9 dt uses the Eulerian |v|+c of the virtual averages and the incircle
 *     diameter 4|T|/perimeter of the virtual triangles (eq. timestep).
 *  R10 the WENO oscillation indicators and weights (eq. weno) are taken per
 *     characteristic field of dF/dQ.n at Q_i, n the direction of the density
 *     gradient of the central-stencil polynomial; the least-squares fits
 *     themselves are linear and use the conserved variables (eq. intConsRec).
 *  R11 positivity safeguards: scaling of w_h at the lattice nodes (density,
 *     then pressure), predictor fallback to w_h (not in the paper).
 *  R12 schedule log: oc_schedule records each element's dt ticks per update
 *     count and replays them, so that runs from perturbed data follow the
 *     base run's schedule (used by the central differences of the adjoint).
 *  R14 Osher-type flux: the path integral of |A_n^V| (eq. osher) by 3-point
 *     Gauss-Legendre quadrature on [0, 1] along the straight path (eq. path).
 *  R16 moving slip wall and start-up: a bc-2 edge mirrors the momentum normal
 *     to it relative to the wall velocity; its nodes move with the wall.
 *     Until t_switch every element takes the global minimum of the local
 *     steps computed with CFL cfl_start, clipped at t_switch (Sec. 3.5).
 *  R17 Kidder boundary state: the outer state of a bc-3 edge is the exact
 *     solution of Sec. 3.4 (eqs. KidderIC, KidderEx, gamma = 2) at the
 *     quadrature point's position and time; the edges are chords of the arcs.
 *  R15 transmissive boundary state: the outer state of a transmissive edge is
 *     the boundary element's cell average at the start of the sweep (not the
 *     inner state at the quadrature point, with which a gas at rest next to
 *     a transmissive boundary grows from roundoff at M >= 1).
 */
#include "aw_oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* Phase marks of the operation-counting build (aw_oracle_count.cpp); no
   effect in this build. */
#ifndef OC_PHASE
#define OC_PHASE(p) ((void)0)
#endif

#define MAXM 3
#define MAXMC 10
#define MAXNT 4
#define MAXNST 40
#define MAXNE 20
#define NSTEN 7

enum { OC_OK = 0, OC_INVALID = -1, OC_BAD_MESH = -2, OC_NONPHYSICAL = -3, OC_DEADLOCK = -4, OC_STATE = -7 };

struct oc_ctx {
  oc_config cfg;
  int M, Mc, Nt, Nst, ne, nit;
  double tick;
  int64_t T;
  char err[256];
  /* --- tables --- */
  int mono[MAXMC][2];
  double lat[MAXMC][2];
  double vinv[MAXMC][MAXMC];      /* phi_s = sum_a vinv[a][s] xi^p eta^q */
  double dub[MAXMC][MAXMC];       /* psi_l = sum_a dub[l][a] xi^p eta^q */
  double Sigma[MAXMC][MAXMC];
  double tau[MAXNT];
  double Kt[MAXNT][MAXNT], Mt[MAXNT][MAXNT], Dtau[MAXNT][MAXNT];
  double Ms[MAXMC][MAXMC];
  double glx[MAXNT], glw[MAXNT];  /* Nt-point Gauss-Legendre on [0,1] */
  int vnode[3];                   /* lattice index of the reference vertices */
  /* space-time Galerkin system restricted to the unknown (tau>0) dofs */
  int nu;
  double* Kuu;  /* LU factors, nu x nu */
  int* piv;
  /* --- mesh --- */
  int64_t nn, ne_;
  int32_t* tri;
  int8_t* bc;
  int8_t* shift;  /* [ne][3][2] */
  int periodic;
  double period[2];
  int64_t Tsw;         /* ticks of the global-step start-up, 0 if none */
  int64_t Ts;          /* sync time in ticks (reading R18): every step is clipped
                          at it and elements stop there; T unless oc_advance_to
                          set an earlier time */
  double wall_speed;   /* |(wall_u, wall_v)| */
  int64_t nedges;
  int32_t* edge_nodes; /* [nedges][2] a,b in the owner's orientation */
  int32_t* edge_elem;  /* [nedges][2] owner (left), right or -1 */
  int8_t* edge_loc;    /* [nedges][2] local edge index in left/right */
  int8_t* edge_bc;     /* bc of boundary edges, -1 interior */
  int32_t* elem_edge;  /* [ne][3] */
  int32_t* nbr;        /* [ne][3] neighbour or -1 */
  int8_t* nbr_shift;   /* [ne][3][2] */
  int64_t* v2e_ptr;    /* node -> elements CSR */
  int32_t* v2e;
  int8_t* v2e_loc;
  int8_t* node_type;   /* 0 free, 1 slide, 2 fixed, 3 moves with the wall */
  double* node_n;      /* [nn][2] wall normal */
  int32_t* sten;       /* [ne][7][ne_max] members, -1 dropped */
  int8_t* sten_shift;  /* [ne][7][ne_max][2] */
  int8_t* sten_ok;     /* [ne][7] */
  int64_t* sw_ptr;
  int32_t* sw;
  /* --- state --- */
  int have_state;
  double *Q, *QM, *HM, *X, *qhat;
  int64_t *t, *dt, *count;
  double* nX;
  int64_t* nt;
  double* xy0;
  double gcl_max;
  double gcl_checked;
  /* --- frozen schedule (record / replay of the dt ticks, reading R12) --- */
  int sched_mode;      /* 0 free, 1 record, 2 replay */
  int64_t sched_k;     /* entries per element: updates 0..sched_k-1 */
  int64_t* sched_log;  /* [ne][sched_k] dt ticks chosen at each update count */
};

static int fail(oc_ctx* c, int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(c->err, sizeof c->err, fmt, ap);
  va_end(ap);
  return code;
}

/* ------------------------------------------------------------------------
 * dense linear algebra (plain textbook forms)
 * ------------------------------------------------------------------------ */

/* LU with partial pivoting of the n x n row-major matrix a, in place. */
static int lu_factor(double* a, int* piv, int n) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(a[i * n + k]) > fabs(a[p * n + k])) p = i;
    piv[k] = p;
    if (a[p * n + k] == 0.0) return -1;
    if (p != k)
      for (int j = 0; j < n; ++j) {
        double tmp = a[k * n + j];
        a[k * n + j] = a[p * n + j];
        a[p * n + j] = tmp;
      }
    for (int i = k + 1; i < n; ++i) {
      a[i * n + k] /= a[k * n + k];
      for (int j = k + 1; j < n; ++j) a[i * n + j] -= a[i * n + k] * a[k * n + j];
    }
  }
  return 0;
}

static void lu_solve(const double* a, const int* piv, int n, double* b) {
  for (int k = 0; k < n; ++k) {
    double tmp = b[k];
    b[k] = b[piv[k]];
    b[piv[k]] = tmp;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) b[i] -= a[i * n + j] * b[j];
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i + 1; j < n; ++j) b[i] -= a[i * n + j] * b[j];
    b[i] /= a[i * n + i];
  }
}

static int invert(const double* a, double* inv, int n) {
  double lu[MAXMC * MAXMC];
  int piv[MAXMC];
  memcpy(lu, a, sizeof(double) * n * n);
  if (lu_factor(lu, piv, n)) return -1;
  for (int j = 0; j < n; ++j) {
    double col[MAXMC];
    for (int i = 0; i < n; ++i) col[i] = (i == j);
    lu_solve(lu, piv, n, col);
    for (int i = 0; i < n; ++i) inv[i * n + j] = col[i];
  }
  return 0;
}

/* Least squares min ||A x - B|| by Householder QR; A is m x n (m >= n),
   B is m x nr; solution written to the first n rows of B. Row-major,
   A has leading dimension n, B leading dimension nr. */
static void householder_lsq(double* A, int m, int n, double* B, int nr) {
  for (int k = 0; k < n; ++k) {
    double norm = 0.0;
    for (int i = k; i < m; ++i) norm += A[i * n + k] * A[i * n + k];
    norm = sqrt(norm);
    if (norm == 0.0) continue;
    double alpha = A[k * n + k] > 0 ? -norm : norm;
    double v[64];
    for (int i = k; i < m; ++i) v[i] = A[i * n + k];
    v[k] -= alpha;
    double vnorm2 = 0.0;
    for (int i = k; i < m; ++i) vnorm2 += v[i] * v[i];
    if (vnorm2 == 0.0) continue;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * A[i * n + j];
      s = 2.0 * s / vnorm2;
      for (int i = k; i < m; ++i) A[i * n + j] -= s * v[i];
    }
    for (int j = 0; j < nr; ++j) {
      double s = 0.0;
      for (int i = k; i < m; ++i) s += v[i] * B[i * nr + j];
      s = 2.0 * s / vnorm2;
      for (int i = k; i < m; ++i) B[i * nr + j] -= s * v[i];
    }
  }
  for (int j = 0; j < nr; ++j)
    for (int i = n - 1; i >= 0; --i) {
      double s = B[i * nr + j];
      for (int k = i + 1; k < n; ++k) s -= A[i * n + k] * B[k * nr + j];
      B[i * nr + j] = s / A[i * n + i];
    }
}

/* ------------------------------------------------------------------------
 * reference-element tables (Sec. 2.2, 2.3)
 * ------------------------------------------------------------------------ */

static double legendre(int n, double x, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    if (dp) *dp = 0.0;
    return 1.0;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  if (dp) *dp = n * (x * p1 - p0) / (x * x - 1.0);
  return p1;
}

/* n-point Gauss-Legendre rule mapped to [0,1] (Newton on P_n). */
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double dp;
      double p = legendre(n, z, &dp);
      double dz = p / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double dp;
    legendre(n, z, &dp);
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

static double ipow(double x, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r *= x;
  return r;
}

static double fact(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

/* Jacobi polynomial P_n^{(a,0)}(x) by the three-term recurrence. */
static double jacobi_a0(int n, double a, double x) {
  if (n == 0) return 1.0;
  double p0 = 1.0, p1 = (a + 1.0) + (a + 2.0) * (x - 1.0) / 2.0;
  for (int k = 2; k <= n; ++k) {
    double c = 2.0 * k + a;
    double a1 = 2.0 * k * (k + a) * (c - 2.0);
    double a2 = (c - 1.0) * (c * (c - 2.0) * x + a * a);
    double a3 = 2.0 * (k + a - 1.0) * (k - 1.0) * c;
    double p2 = (a2 * p1 - a3 * p0) / a1;
    p0 = p1;
    p1 = p2;
  }
  return p1;
}

/* Dubiner's orthogonal basis on T_e = {(0,0),(1,0),(0,1)}:
   psi_{p,q} = P_p(a) ((1-b)/2)^p P_q^{(2p+1,0)}(b), a = 2 xi/(1-eta) - 1,
   b = 2 eta - 1.  P_p(a)(1-eta)^p is evaluated as a homogeneous polynomial
   (scaled Legendre recurrence) so that eta = 1 needs no division. */
static void dubiner_eval(const oc_ctx* c, double xi, double eta, double* out) {
  int l = 0;
  for (int d = 0; d <= c->M; ++d)
    for (int q = 0; q <= d; ++q) {
      int p = d - q;
      double s = 1.0 - eta, z = 2.0 * xi - s;
      double L0 = 1.0, L1 = z, Lp;
      if (p == 0)
        Lp = 1.0;
      else if (p == 1)
        Lp = z;
      else {
        for (int k = 1; k < p; ++k) {
          double L2 = ((2 * k + 1) * z * L1 - k * s * s * L0) / (k + 1);
          L0 = L1;
          L1 = L2;
        }
        Lp = L1;
      }
      out[l++] = Lp * jacobi_a0(q, 2.0 * p + 1.0, 2.0 * eta - 1.0);
    }
}

static void mono_eval(const oc_ctx* c, double xi, double eta, double* m) {
  for (int a = 0; a < c->Mc; ++a) m[a] = ipow(xi, c->mono[a][0]) * ipow(eta, c->mono[a][1]);
}

/* spatial Lagrange basis on the lattice */
static void lagrange_eval(const oc_ctx* c, double xi, double eta, double* phi) {
  double m[MAXMC];
  mono_eval(c, xi, eta, m);
  for (int s = 0; s < c->Mc; ++s) {
    double v = 0.0;
    for (int a = 0; a < c->Mc; ++a) v += c->vinv[a][s] * m[a];
    phi[s] = v;
  }
}

/* temporal Lagrange basis on the Gauss-Lobatto nodes */
static void time_basis(const oc_ctx* c, double tau, double* L) {
  for (int t = 0; t < c->Nt; ++t) {
    double v = 1.0;
    for (int u = 0; u < c->Nt; ++u)
      if (u != t) v *= (tau - c->tau[u]) / (c->tau[t] - c->tau[u]);
    L[t] = v;
  }
}

static void time_basis_deriv(const oc_ctx* c, double tau, double* dL) {
  for (int t = 0; t < c->Nt; ++t) {
    double sum = 0.0;
    for (int k = 0; k < c->Nt; ++k) {
      if (k == t) continue;
      double v = 1.0 / (c->tau[t] - c->tau[k]);
      for (int u = 0; u < c->Nt; ++u)
        if (u != t && u != k) v *= (tau - c->tau[u]) / (c->tau[t] - c->tau[u]);
      sum += v;
    }
    dL[t] = sum;
  }
}

/* Collapsed (Duffy) Gauss rule on T_e: points (s,t) with weights that sum to 1. */
static int duffy_rule(int n, double* s, double* t, double* w) {
  double x[8], wx[8];
  gauss_legendre01(n, x, wx);
  int k = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      s[k] = x[i] * (1.0 - x[j]);
      t[k] = x[j];
      w[k] = 2.0 * wx[i] * wx[j] * (1.0 - x[j]);
      ++k;
    }
  return k;
}

static int build_tables(oc_ctx* c) {
  int M = c->M;
  int a = 0;
  for (int d = 0; d <= M; ++d)
    for (int q = 0; q <= d; ++q) {
      c->mono[a][0] = d - q;
      c->mono[a][1] = q;
      ++a;
    }
  int s = 0;
  for (int j = 0; j <= M; ++j)
    for (int i = 0; i <= M - j; ++i) {
      c->lat[s][0] = (double)i / M;
      c->lat[s][1] = (double)j / M;
      ++s;
    }
  c->vnode[0] = 0;
  c->vnode[1] = M;
  c->vnode[2] = c->Mc - 1;
  double V[MAXMC * MAXMC], Vi[MAXMC * MAXMC];
  for (s = 0; s < c->Mc; ++s) {
    double m[MAXMC];
    mono_eval(c, c->lat[s][0], c->lat[s][1], m);
    for (a = 0; a < c->Mc; ++a) V[s * c->Mc + a] = m[a];
  }
  if (invert(V, Vi, c->Mc)) return -1;
  for (a = 0; a < c->Mc; ++a)
    for (s = 0; s < c->Mc; ++s) c->vinv[a][s] = Vi[a * c->Mc + s];
  /* Dubiner functions in monomial form: interpolate at the lattice */
  for (int l = 0; l < c->Mc; ++l)
    for (a = 0; a < c->Mc; ++a) c->dub[l][a] = 0.0;
  for (s = 0; s < c->Mc; ++s) {
    double psi[MAXMC];
    dubiner_eval(c, c->lat[s][0], c->lat[s][1], psi);
    for (int l = 0; l < c->Mc; ++l)
      for (a = 0; a < c->Mc; ++a) c->dub[l][a] += c->vinv[a][s] * psi[l];
  }
  /* Sigma_lm = sum_{1<=alpha+beta<=M} int_Te d^{ab} psi_l d^{ab} psi_m (exact on monomials) */
  for (int l = 0; l < c->Mc; ++l)
    for (int m = 0; m < c->Mc; ++m) {
      double sum = 0.0;
      for (int al = 0; al <= M; ++al)
        for (int be = 0; al + be <= M; ++be) {
          if (al + be == 0) continue;
          for (int a1 = 0; a1 < c->Mc; ++a1) {
            int p1 = c->mono[a1][0], q1 = c->mono[a1][1];
            if (p1 < al || q1 < be || c->dub[l][a1] == 0.0) continue;
            double c1 = c->dub[l][a1] * fact(p1) / fact(p1 - al) * fact(q1) / fact(q1 - be);
            for (int a2 = 0; a2 < c->Mc; ++a2) {
              int p2 = c->mono[a2][0], q2 = c->mono[a2][1];
              if (p2 < al || q2 < be || c->dub[m][a2] == 0.0) continue;
              double c2 = c->dub[m][a2] * fact(p2) / fact(p2 - al) * fact(q2) / fact(q2 - be);
              int pa = p1 - al + p2 - al, qa = q1 - be + q2 - be;
              sum += c1 * c2 * fact(pa) * fact(qa) / fact(pa + qa + 2);
            }
          }
        }
      c->Sigma[l][m] = sum;
    }
  /* Gauss-Lobatto time nodes on [0,1] */
  if (M == 1) {
    c->tau[0] = 0.0; c->tau[1] = 1.0;
  } else if (M == 2) {
    c->tau[0] = 0.0; c->tau[1] = 0.5; c->tau[2] = 1.0;
  } else {
    c->tau[0] = 0.0; c->tau[1] = 0.5 - sqrt(5.0) / 10.0;
    c->tau[2] = 0.5 + sqrt(5.0) / 10.0; c->tau[3] = 1.0;
  }
  gauss_legendre01(c->Nt, c->glx, c->glw);
  /* K_t, M_t with an (Nt+1)-point Gauss rule (exact) */
  double qx[8], qw[8];
  gauss_legendre01(c->Nt + 1, qx, qw);
  for (int k = 0; k < c->Nt; ++k)
    for (int l = 0; l < c->Nt; ++l) {
      c->Kt[k][l] = 0.0;
      c->Mt[k][l] = 0.0;
    }
  for (int g = 0; g < c->Nt + 1; ++g) {
    double L[MAXNT], dL[MAXNT];
    time_basis(c, qx[g], L);
    time_basis_deriv(c, qx[g], dL);
    for (int k = 0; k < c->Nt; ++k)
      for (int l = 0; l < c->Nt; ++l) {
        c->Kt[k][l] += qw[g] * L[k] * dL[l];
        c->Mt[k][l] += qw[g] * L[k] * L[l];
      }
  }
  for (int t = 0; t < c->Nt; ++t) {
    double dL[MAXNT];
    time_basis_deriv(c, c->tau[t], dL);
    for (int u = 0; u < c->Nt; ++u) c->Dtau[t][u] = dL[u];
  }
  /* spatial mass matrix of the Lagrange basis, exact Duffy rule */
  double ps[64], pt[64], pw[64];
  int nq = duffy_rule(M + 2, ps, pt, pw);
  for (int i = 0; i < c->Mc; ++i)
    for (int j = 0; j < c->Mc; ++j) c->Ms[i][j] = 0.0;
  for (int g = 0; g < nq; ++g) {
    double phi[MAXMC];
    lagrange_eval(c, ps[g], pt[g], phi);
    for (int i = 0; i < c->Mc; ++i)
      for (int j = 0; j < c->Mc; ++j) c->Ms[i][j] += 0.5 * pw[g] * phi[i] * phi[j];
  }
  /* space-time matrices K_tau = <theta_k, d_tau theta_l>, M = <theta_k, theta_l>
     (eq. Ktau) restricted to rows and columns of the unknown tau>0 dofs; the
     LU factors of K_uu are kept. */
  c->nu = c->Mc * c->M;
  c->Kuu = (double*)malloc(sizeof(double) * c->nu * c->nu);
  c->piv = (int*)malloc(sizeof(int) * c->nu);
  for (int k = 0; k < c->nu; ++k)
    for (int l = 0; l < c->nu; ++l) {
      int tk = 1 + k / c->Mc, sk = k % c->Mc, tl = 1 + l / c->Mc, sl = l % c->Mc;
      c->Kuu[k * c->nu + l] = c->Ms[sk][sl] * c->Kt[tk][tl];
    }
  if (lu_factor(c->Kuu, c->piv, c->nu)) return -1;
  return 0;
}

/* ------------------------------------------------------------------------
 * small geometric helpers
 * ------------------------------------------------------------------------ */

static double tri_area(const double* X) {
  return 0.5 * ((X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0]));
}

static double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

static void corner(const oc_ctx* c, int64_t i, int k, const double* nodeX, double* out) {
  int32_t n = c->tri[i * 3 + k];
  out[0] = nodeX[2 * n];
  out[1] = nodeX[2 * n + 1];
  if (c->periodic) {
    out[0] += c->shift[(i * 3 + k) * 2] * c->period[0];
    out[1] += c->shift[(i * 3 + k) * 2 + 1] * c->period[1];
  }
}

/* ------------------------------------------------------------------------
 * mesh pre-processing: edges, Voronoi sets, stencils (Sec. 2.2, R3)
 * ------------------------------------------------------------------------ */

typedef struct {
  double d2;
  int32_t j;
  int8_t sx, sy;
} cand_t;

static int cand_cmp(const void* a, const void* b) {
  const cand_t* x = (const cand_t*)a;
  const cand_t* y = (const cand_t*)b;
  if (x->d2 < y->d2) return -1;
  if (x->d2 > y->d2) return 1;
  return (x->j > y->j) - (x->j < y->j);
}

/* centroid offset of j seen from i at t=0, with the nearest periodic image */
static void rel_offset(const oc_ctx* c, const double* cen, int64_t i, int64_t j, double* d, int* sx, int* sy) {
  double dx = cen[2 * j] - cen[2 * i];
  double dy = cen[2 * j + 1] - cen[2 * i + 1];
  int ix = 0, iy = 0;
  if (c->periodic) {
    /* a zero period component: not periodic in that direction */
    if (c->period[0] > 0.0) ix = -(int)floor(dx / c->period[0] + 0.5);
    if (c->period[1] > 0.0) iy = -(int)floor(dy / c->period[1] + 0.5);
    dx = dx + ix * c->period[0];
    dy = dy + iy * c->period[1];
  }
  d[0] = dx;
  d[1] = dy;
  *sx = ix;
  *sy = iy;
}

/* vertex-neighbour layers 0..depth around element i */
static int collect_layers(const oc_ctx* c, int64_t i, int depth, int32_t* mark, int32_t stamp, int32_t* out, int cap) {
  int n = 0, begin = 0;
  out[n++] = (int32_t)i;
  mark[i] = stamp;
  for (int d = 0; d < depth; ++d) {
    int end = n;
    for (int q = begin; q < end; ++q) {
      int32_t e = out[q];
      for (int k = 0; k < 3; ++k) {
        int32_t node = c->tri[e * 3 + k];
        for (int64_t p = c->v2e_ptr[node]; p < c->v2e_ptr[node + 1]; ++p) {
          int32_t j = c->v2e[p];
          if (mark[j] == stamp) continue;
          mark[j] = stamp;
          if (n < cap) out[n++] = j;
        }
      }
    }
    begin = end;
  }
  return n;
}

static int build_mesh(oc_ctx* c, const double* xy) {
  int64_t ne = c->ne_, nn = c->nn;
  /* node -> element lists, ascending element index */
  c->v2e_ptr = (int64_t*)calloc(nn + 1, sizeof(int64_t));
  for (int64_t i = 0; i < ne; ++i)
    for (int k = 0; k < 3; ++k) c->v2e_ptr[c->tri[i * 3 + k] + 1]++;
  for (int64_t n = 0; n < nn; ++n) c->v2e_ptr[n + 1] += c->v2e_ptr[n];
  c->v2e = (int32_t*)malloc(sizeof(int32_t) * 3 * ne);
  c->v2e_loc = (int8_t*)malloc(3 * ne);
  int64_t* fill = (int64_t*)calloc(nn, sizeof(int64_t));
  for (int64_t i = 0; i < ne; ++i)
    for (int k = 0; k < 3; ++k) {
      int32_t n = c->tri[i * 3 + k];
      int64_t p = c->v2e_ptr[n] + fill[n]++;
      c->v2e[p] = (int32_t)i;
      c->v2e_loc[p] = (int8_t)k;
    }
  free(fill);
  /* corners at t=0, areas, centroids */
  double* cen = (double*)malloc(sizeof(double) * 2 * ne);
  for (int64_t i = 0; i < ne; ++i) {
    double X[6];
    for (int k = 0; k < 3; ++k) corner(c, i, k, xy, X + 2 * k);
    if (!(tri_area(X) > 0.0)) {
      free(cen);
      return fail(c, OC_BAD_MESH, "element %lld is not counter-clockwise", (long long)i);
    }
    cen[2 * i] = (X[0] + X[2] + X[4]) / 3.0;
    cen[2 * i + 1] = (X[1] + X[3] + X[5]) / 3.0;
  }
  /* edges: twin search through the Voronoi set of the first node */
  c->nbr = (int32_t*)malloc(sizeof(int32_t) * 3 * ne);
  int8_t* nbr_loc = (int8_t*)malloc(3 * ne);
  for (int64_t i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      int32_t a = c->tri[i * 3 + e], b = c->tri[i * 3 + (e + 1) % 3];
      int found = 0;
      c->nbr[i * 3 + e] = -1;
      nbr_loc[i * 3 + e] = -1;
      for (int64_t p = c->v2e_ptr[a]; p < c->v2e_ptr[a + 1]; ++p) {
        int32_t j = c->v2e[p];
        if (j == i) continue;
        for (int f = 0; f < 3; ++f)
          if (c->tri[j * 3 + f] == b && c->tri[j * 3 + (f + 1) % 3] == a) {
            c->nbr[i * 3 + e] = j;
            nbr_loc[i * 3 + e] = (int8_t)f;
            ++found;
          }
      }
      if (found > 1) {
        free(cen); free(nbr_loc);
        return fail(c, OC_BAD_MESH, "edge of element %lld is non-manifold", (long long)i);
      }
      if (found == 0 && c->bc[i * 3 + e] < 0) {
        free(cen); free(nbr_loc);
        return fail(c, OC_BAD_MESH, "boundary edge of element %lld has no boundary tag", (long long)i);
      }
    }
  /* canonical edge numbering: element order, owner = lower element index */
  c->elem_edge = (int32_t*)malloc(sizeof(int32_t) * 3 * ne);
  c->edge_nodes = (int32_t*)malloc(sizeof(int32_t) * 2 * 3 * ne);
  c->edge_elem = (int32_t*)malloc(sizeof(int32_t) * 2 * 3 * ne);
  c->edge_loc = (int8_t*)malloc(2 * 3 * ne);
  c->edge_bc = (int8_t*)malloc(3 * ne);
  int64_t ned = 0;
  for (int64_t i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      int32_t j = c->nbr[i * 3 + e];
      if (j >= 0 && j < i) {
        c->elem_edge[i * 3 + e] = c->elem_edge[j * 3 + nbr_loc[i * 3 + e]];
        continue;
      }
      c->elem_edge[i * 3 + e] = (int32_t)ned;
      c->edge_nodes[2 * ned] = c->tri[i * 3 + e];
      c->edge_nodes[2 * ned + 1] = c->tri[i * 3 + (e + 1) % 3];
      c->edge_elem[2 * ned] = (int32_t)i;
      c->edge_elem[2 * ned + 1] = j;
      c->edge_loc[2 * ned] = (int8_t)e;
      c->edge_loc[2 * ned + 1] = j >= 0 ? nbr_loc[i * 3 + e] : -1;
      c->edge_bc[ned] = j >= 0 ? -1 : c->bc[i * 3 + e];
      ++ned;
    }
  c->nedges = ned;
  free(nbr_loc);
  /* neighbour image shifts */
  c->nbr_shift = (int8_t*)calloc(6 * ne, 1);
  for (int64_t i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      int32_t j = c->nbr[i * 3 + e];
      if (j < 0) continue;
      double d[2];
      int sx, sy;
      rel_offset(c, cen, i, j, d, &sx, &sy);
      c->nbr_shift[(i * 3 + e) * 2] = (int8_t)sx;
      c->nbr_shift[(i * 3 + e) * 2 + 1] = (int8_t)sy;
    }
  /* wall constraints of nodes */
  c->node_type = (int8_t*)calloc(nn, 1);
  c->node_n = (double*)calloc(2 * nn, sizeof(double));
  for (int64_t ed = 0; ed < ned; ++ed) {
    if (c->edge_bc[ed] != 0) continue;
    int32_t i = c->edge_elem[2 * ed];
    int e = c->edge_loc[2 * ed];
    double A[2], B[2];
    corner(c, i, e, xy, A);
    corner(c, i, (e + 1) % 3, xy, B);
    double dx = B[0] - A[0], dy = B[1] - A[1];
    double len = sqrt(dx * dx + dy * dy);
    double n0 = dy / len, n1 = -dx / len;
    for (int q = 0; q < 2; ++q) {
      int32_t node = c->edge_nodes[2 * ed + q];
      if (c->node_type[node] == 0) {
        c->node_type[node] = 1;
        c->node_n[2 * node] = n0;
        c->node_n[2 * node + 1] = n1;
      } else if (c->node_type[node] == 1) {
        if (fabs(cross2(c->node_n[2 * node], c->node_n[2 * node + 1], n0, n1)) > 1e-8) c->node_type[node] = 2;
      }
    }
  }
  /* nodes of moving walls move with the wall (R16) */
  for (int64_t ed = 0; ed < ned; ++ed)
    if (c->edge_bc[ed] == 2)
      for (int q = 0; q < 2; ++q) c->node_type[c->edge_nodes[2 * ed + q]] = 3;
  /* stencils */
  int ne_s = c->ne;
  c->sten = (int32_t*)malloc(sizeof(int32_t) * ne * NSTEN * ne_s);
  c->sten_shift = (int8_t*)calloc((size_t)ne * NSTEN * ne_s * 2, 1);
  c->sten_ok = (int8_t*)calloc(ne * NSTEN, 1);
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * ne);
  for (int64_t i = 0; i < ne; ++i) mark[i] = -1;
  int cap = 4096;
  int32_t* lay = (int32_t*)malloc(sizeof(int32_t) * cap);
  cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * cap);
  int32_t stamp = 0;
  for (int64_t i = 0; i < ne; ++i) {
    double Xi[6];
    for (int k = 0; k < 3; ++k) corner(c, i, k, xy, Xi + 2 * k);
    double cx = cen[2 * i], cy = cen[2 * i + 1];
    int32_t* S = c->sten + i * NSTEN * ne_s;
    int8_t* SS = c->sten_shift + i * NSTEN * ne_s * 2;
    for (int q = 0; q < NSTEN * ne_s; ++q) S[q] = -1;
    /* central stencil */
    int n = collect_layers(c, i, c->M + 1, mark, stamp++, lay, cap);
    for (int q = 0; q < n; ++q) {
      double d[2];
      int sx, sy;
      rel_offset(c, cen, i, lay[q], d, &sx, &sy);
      cand[q].d2 = d[0] * d[0] + d[1] * d[1];
      cand[q].j = lay[q];
      cand[q].sx = (int8_t)sx;
      cand[q].sy = (int8_t)sy;
    }
    qsort(cand, n, sizeof(cand_t), cand_cmp);
    if (n < ne_s) {
      free(cen); free(mark); free(lay); free(cand);
      return fail(c, OC_BAD_MESH, "element %lld: only %d candidates for the central stencil", (long long)i, n);
    }
    for (int q = 0; q < ne_s; ++q) {
      S[q] = cand[q].j;
      SS[2 * q] = cand[q].sx;
      SS[2 * q + 1] = cand[q].sy;
    }
    c->sten_ok[i * NSTEN] = 1;
    /* sector stencils */
    n = collect_layers(c, i, c->M + 2, mark, stamp++, lay, cap);
    for (int q = 0; q < n; ++q) {
      double d[2];
      int sx, sy;
      rel_offset(c, cen, i, lay[q], d, &sx, &sy);
      cand[q].d2 = d[0] * d[0] + d[1] * d[1];
      cand[q].j = lay[q];
      cand[q].sx = (int8_t)sx;
      cand[q].sy = (int8_t)sy;
    }
    qsort(cand, n, sizeof(cand_t), cand_cmp);
    for (int s = 1; s < NSTEN; ++s) {
      int e = (s - 1) % 3;
      int reverse = s >= 4;
      double ax = Xi[2 * e] - cx, ay = Xi[2 * e + 1] - cy;
      double bx = Xi[2 * ((e + 1) % 3)] - cx, by = Xi[2 * ((e + 1) % 3) + 1] - cy;
      int m = 0;
      S[s * ne_s + m++] = (int32_t)i;
      for (int q = 0; q < n && m < ne_s; ++q) {
        if (cand[q].j == i) continue;
        double dx = cen[2 * cand[q].j] - cx + cand[q].sx * (c->periodic ? c->period[0] : 0.0);
        double dy = cen[2 * cand[q].j + 1] - cy + cand[q].sy * (c->periodic ? c->period[1] : 0.0);
        double alpha = cross2(dx, dy, bx, by);
        double beta = cross2(ax, ay, dx, dy);
        int in = reverse ? (alpha <= 0.0 && beta <= 0.0) : (alpha >= 0.0 && beta >= 0.0);
        if (!in) continue;
        S[s * ne_s + m] = cand[q].j;
        SS[(s * ne_s + m) * 2] = cand[q].sx;
        SS[(s * ne_s + m) * 2 + 1] = cand[q].sy;
        ++m;
      }
      if (m == ne_s)
        c->sten_ok[i * NSTEN + s] = 1;
      else
        for (int q = 0; q < ne_s; ++q) S[s * ne_s + q] = -1;
    }
  }
  free(lay);
  free(cand);
  /* total stencil S^W: stencils, edge neighbours, Voronoi sets of the vertices;
     then closed under symmetry (Sec. 2.2) */
  int64_t* cnt = (int64_t*)calloc(ne + 1, sizeof(int64_t));
  int32_t** lists = (int32_t**)malloc(sizeof(int32_t*) * ne);
  int* lsz = (int*)calloc(ne, sizeof(int));
  int* lcap = (int*)calloc(ne, sizeof(int));
  for (int64_t i = 0; i < ne; ++i) {
    lcap[i] = 64;
    lists[i] = (int32_t*)malloc(sizeof(int32_t) * lcap[i]);
  }
#define ADD(i_, j_)                                                        \
  do {                                                                     \
    if (lsz[i_] == lcap[i_]) {                                             \
      lcap[i_] *= 2;                                                       \
      lists[i_] = (int32_t*)realloc(lists[i_], sizeof(int32_t) * lcap[i_]); \
    }                                                                      \
    lists[i_][lsz[i_]++] = (j_);                                           \
  } while (0)
  for (int64_t i = 0; i < ne; ++i) mark[i] = -1;
  stamp = 0;
  for (int64_t i = 0; i < ne; ++i) {
    ++stamp;
    int32_t* S = c->sten + i * NSTEN * ne_s;
    for (int q = 0; q < NSTEN * ne_s; ++q)
      if (S[q] >= 0 && mark[S[q]] != stamp) {
        mark[S[q]] = stamp;
        ADD(i, S[q]);
      }
    for (int e = 0; e < 3; ++e) {
      int32_t j = c->nbr[i * 3 + e];
      if (j >= 0 && mark[j] != stamp) {
        mark[j] = stamp;
        ADD(i, j);
      }
    }
    for (int k = 0; k < 3; ++k) {
      int32_t node = c->tri[i * 3 + k];
      for (int64_t p = c->v2e_ptr[node]; p < c->v2e_ptr[node + 1]; ++p) {
        int32_t j = c->v2e[p];
        if (mark[j] != stamp) {
          mark[j] = stamp;
          ADD(i, j);
        }
      }
    }
  }
  /* symmetric closure: add i to S^W_j for every j in S^W_i */
  int* base = (int*)malloc(sizeof(int) * ne);
  for (int64_t i = 0; i < ne; ++i) base[i] = lsz[i];
  for (int64_t i = 0; i < ne; ++i)
    for (int q = 0; q < base[i]; ++q) {
      int32_t j = lists[i][q];
      ADD(j, (int32_t)i);
    }
  free(base);
  /* sort and deduplicate */
  for (int64_t i = 0; i < ne; ++i) {
    int32_t* L = lists[i];
    int n = lsz[i];
    for (int a1 = 1; a1 < n; ++a1) {
      int32_t v = L[a1];
      int b1 = a1 - 1;
      while (b1 >= 0 && L[b1] > v) {
        L[b1 + 1] = L[b1];
        --b1;
      }
      L[b1 + 1] = v;
    }
    int m = 0;
    for (int q = 0; q < n; ++q)
      if (m == 0 || L[m - 1] != L[q]) L[m++] = L[q];
    lsz[i] = m;
    cnt[i + 1] = cnt[i] + m;
  }
  c->sw_ptr = cnt;
  c->sw = (int32_t*)malloc(sizeof(int32_t) * (cnt[ne] > 0 ? cnt[ne] : 1));
  for (int64_t i = 0; i < ne; ++i) {
    memcpy(c->sw + cnt[i], lists[i], sizeof(int32_t) * lsz[i]);
    free(lists[i]);
  }
#undef ADD
  free(lists);
  free(lsz);
  free(lcap);
  free(mark);
  free(cen);
  return OC_OK;
}

/* ------------------------------------------------------------------------
 * evaluation of the predictor (eq. thetaSol) and the Euler system (eq. eulerTerms)
 * ------------------------------------------------------------------------ */

static void eval_qh(const oc_ctx* c, const double* qh, double xi, double eta, double tau, double* q) {
  double phi[MAXMC], L[MAXNT];
  lagrange_eval(c, xi, eta, phi);
  time_basis(c, tau, L);
  for (int v = 0; v < 4; ++v) q[v] = 0.0;
  for (int t = 0; t < c->Nt; ++t)
    for (int s = 0; s < c->Mc; ++s) {
      double b = phi[s] * L[t];
      for (int v = 0; v < 4; ++v) q[v] += b * qh[(t * c->Mc + s) * 4 + v];
    }
}

static double pressure(const oc_ctx* c, const double* q) {
  return (c->cfg.gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

static void euler_flux(const oc_ctx* c, const double* q, double* f, double* g) {
  double u = q[1] / q[0], v = q[2] / q[0], p = pressure(c, q);
  f[0] = q[1];
  f[1] = q[1] * u + p;
  f[2] = q[1] * v;
  f[3] = u * (q[3] + p);
  g[0] = q[2];
  g[1] = q[2] * u;
  g[2] = q[2] * v + p;
  g[3] = v * (q[3] + p);
}

/* mesh velocity V = v at a vertex of element j: integral over [ta,tb] of
   V_h(xi_vertex, tau) (eq. NodesVel), exact Gauss-Legendre in tau */
static void vertex_velocity_integral(const oc_ctx* c, const double* qh, int k, double ta, double tb, double* out) {
  out[0] = out[1] = 0.0;
  if (tb == ta || c->cfg.mesh_velocity == 1) return;
  int s = c->vnode[k];
  for (int g = 0; g < c->Nt; ++g) {
    double tau = ta + (tb - ta) * c->glx[g];
    double L[MAXNT];
    time_basis(c, tau, L);
    double u = 0.0, v = 0.0;
    for (int t = 0; t < c->Nt; ++t) {
      const double* q = qh + (t * c->Mc + s) * 4;
      u += L[t] * (q[1] / q[0]);
      v += L[t] * (q[2] / q[0]);
    }
    out[0] += (tb - ta) * c->glw[g] * u;
    out[1] += (tb - ta) * c->glw[g] * v;
  }
}

/* Rusanov-type ALE flux (eq. rusanov) through the area-weighted space-time
   normal n = (n_x, n_y, n_t), oriented from the left (-) to the right (+)
   state.  The largest eigenvalue of A_n^V scaled by |n_xy| is
   |v.n_xy + n_t| + c |n_xy|, since V.n |n_xy| = -n_t. */
static void rusanov(const oc_ctx* c, const double* qm, const double* qp, const double* n, double* F) {
  double fm[4], gm[4], fp[4], gp[4];
  euler_flux(c, qm, fm, gm);
  euler_flux(c, qp, fp, gp);
  double nxy = sqrt(n[0] * n[0] + n[1] * n[1]);
  double cm = sqrt(c->cfg.gamma * pressure(c, qm) / qm[0]);
  double cp = sqrt(c->cfg.gamma * pressure(c, qp) / qp[0]);
  double lm = fabs(qm[1] / qm[0] * n[0] + qm[2] / qm[0] * n[1] + n[2]) + cm * nxy;
  double lp = fabs(qp[1] / qp[0] * n[0] + qp[2] / qp[0] * n[1] + n[2]) + cp * nxy;
  double smax = lm > lp ? lm : lp;
  for (int v = 0; v < 4; ++v) {
    double Fm = fm[v] * n[0] + gm[v] * n[1] + qm[v] * n[2];
    double Fp = fp[v] * n[0] + gp[v] * n[1] + qp[v] * n[2];
    F[v] = 0.5 * (Fm + Fp) - 0.5 * smax * (qp[v] - qm[v]);
  }
}

/* Osher-type ALE flux (eq. osher) on the straight-line path Psi(s) = q- +
   s (q+ - q-) (eq. path).  The path integral of |A_n^V(Psi(s))| is taken by
   3-point Gauss-Legendre quadrature on [0, 1] (reading R14).  At each node
   |A| = R |Lambda| R^-1: the eigenvalues of the ALE Jacobian of F.n_xy + q n_t
   are |n_xy| (u_n - c, u_n, u_n, u_n + c) + n_t, and R holds the
   eigenvectors of dF/dQ.n with n = n_xy / |n_xy| (x if n_xy vanishes);
   R^-1 is the numerical inverse. */
static void osher(const oc_ctx* c, const double* qm, const double* qp, const double* n, double* F) {
  double fm[4], gm[4], fp[4], gp[4];
  euler_flux(c, qm, fm, gm);
  euler_flux(c, qp, fp, gp);
  double nxy = sqrt(n[0] * n[0] + n[1] * n[1]);
  double nx = 1.0, ny = 0.0;
  if (nxy > 0.0) {
    nx = n[0] / nxy;
    ny = n[1] / nxy;
  }
  double dq[4], D[4] = {0.0, 0.0, 0.0, 0.0};
  for (int v = 0; v < 4; ++v) dq[v] = qp[v] - qm[v];
  const double r15 = sqrt(15.0) / 10.0;
  const double sp[3] = {0.5 - r15, 0.5, 0.5 + r15}, sw[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
  for (int gq = 0; gq < 3; ++gq) {
    double q[4];
    for (int v = 0; v < 4; ++v) q[v] = qm[v] + sp[gq] * dq[v];
    double g = c->cfg.gamma, rho = q[0], u = q[1] / rho, v = q[2] / rho, p = pressure(c, q);
    double a = sqrt(g * p / rho), H = (q[3] + p) / rho, un = u * nx + v * ny, ut = -u * ny + v * nx;
    double R[16] = {1.0, 1.0, 0.0, 1.0,
                    u - a * nx, u, -ny, u + a * nx,
                    v - a * ny, v, nx, v + a * ny,
                    H - a * un, 0.5 * (u * u + v * v), ut, H + a * un};
    double Rinv[16];
    invert(R, Rinv, 4);
    double lam[4] = {nxy * (un - a) + n[2], nxy * un + n[2], nxy * un + n[2], nxy * (un + a) + n[2]};
    double w[4];
    for (int k = 0; k < 4; ++k) {
      double acc = 0.0;
      for (int j = 0; j < 4; ++j) acc += Rinv[4 * k + j] * dq[j];
      w[k] = fabs(lam[k]) * acc;
    }
    for (int i = 0; i < 4; ++i) {
      double acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += R[4 * i + k] * w[k];
      D[i] += sw[gq] * acc;
    }
  }
  for (int v = 0; v < 4; ++v) {
    double Fm = fm[v] * n[0] + gm[v] * n[1] + qm[v] * n[2];
    double Fp = fp[v] * n[0] + gp[v] * n[1] + qp[v] * n[2];
    F[v] = 0.5 * (Fm + Fp) - 0.5 * D[v];
  }
}

/* the numerical flux of the configuration (eq. rusanov or eq. osher) */
static void num_flux(const oc_ctx* c, const double* qm, const double* qp, const double* n, double* F) {
  if (c->cfg.flux == 1) osher(c, qm, qp, n, F);
  else rusanov(c, qm, qp, n, F);
}

/* Exact state of the Kidder compression (Sec. 3.4) at (x, y, t): a particle
   that starts at radius r is at h(t) r with h = sqrt(1 - t^2/tau^2); the
   density is rho0(r)/h^2 with rho0^(gamma-1) linear in r^2 between
   rho_i0^(gamma-1) at r_i0 and rho_e0^(gamma-1) at r_e0 (eq. KidderIC), the
   velocity h'(t) r along the radius, the pressure s0 rho^gamma.  tau is the
   focalisation time sqrt((gamma-1)/2 (r_e0^2 - r_i0^2)/(c_e0^2 - c_i0^2)). */
static void kidder_state(const oc_ctx* c, double x, double y, double t, double* q) {
  const double* k = c->cfg.kidder;
  double g = c->cfg.gamma, ri = k[0], re = k[1], s0 = k[4];
  double ai = pow(k[2], g - 1.0), ae = pow(k[3], g - 1.0);
  double ci2 = g * s0 * ai, ce2 = g * s0 * ae;
  double tau2 = 0.5 * (g - 1.0) * (re * re - ri * ri) / (ce2 - ci2);
  double h = sqrt(1.0 - t * t / tau2), dh = -t / (tau2 * h);
  double R = sqrt(x * x + y * y), r = R / h;
  double w = (r * r - ri * ri) / (re * re - ri * ri);
  double rho = pow((1.0 - w) * ai + w * ae, 1.0 / (g - 1.0)) / (h * h);
  double u = dh / h * x, v = dh / h * y;
  double p = s0 * pow(rho, g);
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

static void boundary_state(const oc_ctx* c, int bc, const double* q, const double* n, double* qb) {
  for (int v = 0; v < 4; ++v) qb[v] = q[v];
  if (bc == 0 || bc == 2) {
    /* mirror the momentum normal to the wall, relative to the wall's velocity */
    double wu = bc == 2 ? c->cfg.wall_u : 0.0, wv = bc == 2 ? c->cfg.wall_v : 0.0;
    double nn = n[0] * n[0] + n[1] * n[1];
    if (nn > 0.0) {
      double mn = ((q[1] - q[0] * wu) * n[0] + (q[2] - q[0] * wv) * n[1]) / nn;
      qb[1] = q[1] - 2.0 * mn * n[0];
      qb[2] = q[2] - 2.0 * mn * n[1];
      /* same internal energy: the mirrored momentum of a moving wall has
         another kinetic energy */
      if (bc == 2) qb[3] = q[3] + 0.5 * (qb[1] * qb[1] + qb[2] * qb[2] - q[1] * q[1] - q[2] * q[2]) / q[0];
    }
  }
}

/* ------------------------------------------------------------------------
 * virtual data (eqs. virtGeom, virtCellaverage; R5)
 * ------------------------------------------------------------------------ */

/* virtual vertices (own frame of j) and average of j at time ti (ticks) */
static void virtual_data(const oc_ctx* c, int64_t j, int64_t ti, double* Xv, double* Qv) {
  const double* Xj = c->X + 6 * j;
  if (c->t[j] == ti || c->dt[j] == 0) {
    memcpy(Xv, Xj, sizeof(double) * 6);
    memcpy(Qv, c->Q + 4 * j, sizeof(double) * 4);
    return;
  }
  double taus = (double)(ti - c->t[j]) / (double)c->dt[j];
  double dtj = (double)c->dt[j] * c->tick;
  const double* qh = c->qhat + (size_t)j * c->Nst * 4;
  for (int k = 0; k < 3; ++k) {
    double I[2];
    vertex_velocity_integral(c, qh, k, 0.0, taus, I);
    Xv[2 * k] = Xj[2 * k] + dtj * I[0];
    Xv[2 * k + 1] = Xj[2 * k + 1] + dtj * I[1];
  }
  double ps[64], pt[64], pw[64];
  int nq = duffy_rule(c->Nt, ps, pt, pw);
  for (int v = 0; v < 4; ++v) Qv[v] = 0.0;
  for (int g = 0; g < nq; ++g) {
    double q[4];
    eval_qh(c, qh, ps[g], pt[g], taus, q);
    for (int v = 0; v < 4; ++v) Qv[v] += pw[g] * q[v];
  }
}

/* ------------------------------------------------------------------------
 * WENO reconstruction (eqs. intConsRec, weno; R4)
 * ------------------------------------------------------------------------ */

/* reference coordinates in the frame of triangle X */
static void to_reference(const double* X, double x, double y, double* xi, double* eta) {
  double a = X[2] - X[0], b = X[4] - X[0], cc = X[3] - X[1], d = X[5] - X[1];
  double det = a * d - b * cc;
  double rx = x - X[0], ry = y - X[1];
  *xi = (d * rx - b * ry) / det;
  *eta = (-cc * rx + a * ry) / det;
}

/* modal coefficients w[l][v] of the WENO polynomial of element i at its current time */
static void reconstruct(const oc_ctx* c, int64_t i, double* w) {
  int Mc = c->Mc, ne_s = c->ne, n = Mc - 1, m = ne_s - 1;
  const double* Xi = c->X + 6 * i;
  const double* Qi = c->Q + 4 * i;
  double ps[64], pt[64], pw[64];
  int nq = duffy_rule(c->Nt, ps, pt, pw);
  double ws[NSTEN][MAXMC][4], sigma[NSTEN][4];
  int ok[NSTEN];
  for (int s = 0; s < NSTEN; ++s) {
    ok[s] = c->sten_ok[i * NSTEN + s];
    if (!ok[s]) continue;
    double A[MAXNE * MAXMC], B[MAXNE * 4];
    for (int r = 0; r < m; ++r) {
      int q = s * ne_s + 1 + r;
      int32_t j = c->sten[i * NSTEN * ne_s + q];
      double Xv[6], Qv[4];
      virtual_data(c, j, c->t[i], Xv, Qv);
      if (c->periodic)
        for (int k = 0; k < 3; ++k) {
          Xv[2 * k] += c->sten_shift[(i * NSTEN * ne_s + q) * 2] * c->period[0];
          Xv[2 * k + 1] += c->sten_shift[(i * NSTEN * ne_s + q) * 2 + 1] * c->period[1];
        }
      for (int l = 1; l < Mc; ++l) A[r * n + l - 1] = 0.0;
      for (int g = 0; g < nq; ++g) {
        double x = Xv[0] + (Xv[2] - Xv[0]) * ps[g] + (Xv[4] - Xv[0]) * pt[g];
        double y = Xv[1] + (Xv[3] - Xv[1]) * ps[g] + (Xv[5] - Xv[1]) * pt[g];
        double xi, eta, psi[MAXMC];
        to_reference(Xi, x, y, &xi, &eta);
        dubiner_eval(c, xi, eta, psi);
        for (int l = 1; l < Mc; ++l) A[r * n + l - 1] += pw[g] * psi[l];
      }
      for (int v = 0; v < 4; ++v) B[r * 4 + v] = Qv[v] - Qi[v];
    }
    householder_lsq(A, m, n, B, 4);
    for (int v = 0; v < 4; ++v) {
      ws[s][0][v] = Qi[v];
      for (int l = 1; l < Mc; ++l) ws[s][l][v] = B[(l - 1) * 4 + v];
    }
  }
  /* R10: the nonlinear weights act on characteristic fields.  The
     direction n is that of the density gradient of the central-stencil
     polynomial at the centroid of T_i (x if it vanishes); R and L = R^-1 are
     the eigenvectors of dF/dQ.n at Q_i. */
  double gx = 0.0, gy = 0.0;
  {
    double dpsi_dxi[MAXMC] = {0}, dpsi_deta[MAXMC] = {0};
    double cx = 1.0 / 3.0, cy = 1.0 / 3.0;
    for (int l = 1; l < Mc; ++l)
      for (int a = 0; a < Mc; ++a) {
        int p = c->mono[a][0], q = c->mono[a][1];
        if (p > 0) dpsi_dxi[l] += c->dub[l][a] * p * ipow(cx, p - 1) * ipow(cy, q);
        if (q > 0) dpsi_deta[l] += c->dub[l][a] * q * ipow(cx, p) * ipow(cy, q - 1);
      }
    double rxi = 0.0, reta = 0.0;
    for (int l = 1; l < Mc; ++l) {
      rxi += dpsi_dxi[l] * ws[0][l][0];
      reta += dpsi_deta[l] * ws[0][l][0];
    }
    /* grad_x rho = J^-T grad_xi rho, J = [[x1-x0, x2-x0],[y1-y0, y2-y0]] */
    double a = Xi[2] - Xi[0], b = Xi[4] - Xi[0], cc = Xi[3] - Xi[1], d = Xi[5] - Xi[1];
    double det = a * d - b * cc;
    gx = (d * rxi - cc * reta) / det;
    gy = (-b * rxi + a * reta) / det;
  }
  double gn = sqrt(gx * gx + gy * gy);
  double nx = 1.0, ny = 0.0;
  if (gn > 0.0) {
    nx = gx / gn;
    ny = gy / gn;
  }
  double R[16], Linv[16];
  {
    double g = c->cfg.gamma, rho = Qi[0], u = Qi[1] / rho, v = Qi[2] / rho, p = pressure(c, Qi);
    double a = sqrt(g * p / rho), H = (Qi[3] + p) / rho, un = u * nx + v * ny, ut = -u * ny + v * nx;
    double Rm[16] = {1.0, 1.0, 0.0, 1.0,
                     u - a * nx, u, -ny, u + a * nx,
                     v - a * ny, v, nx, v + a * ny,
                     H - a * un, 0.5 * (u * u + v * v), ut, H + a * un};
    memcpy(R, Rm, sizeof Rm);
    invert(R, Linv, 4);
  }
  double wc[NSTEN][MAXMC][4];
  for (int s = 0; s < NSTEN; ++s) {
    if (!ok[s]) continue;
    for (int l = 1; l < Mc; ++l)
      for (int r = 0; r < 4; ++r) {
        double acc = 0.0;
        for (int k = 0; k < 4; ++k) acc += Linv[r * 4 + k] * ws[s][l][k];
        wc[s][l][r] = acc;
      }
    for (int r = 0; r < 4; ++r) {
      double sg = 0.0;
      for (int l = 1; l < Mc; ++l)
        for (int k = 1; k < Mc; ++k) sg += c->Sigma[l][k] * wc[s][l][r] * wc[s][k][r];
      sigma[s][r] = sg;
    }
  }
  double wchar[MAXMC][4];
  for (int r = 0; r < 4; ++r) {
    double om[NSTEN], tot = 0.0;
    for (int s = 0; s < NSTEN; ++s) {
      om[s] = 0.0;
      if (!ok[s]) continue;
      double lam = s == 0 ? 1e5 : 1.0;
      om[s] = lam / pow(sigma[s][r] + 1e-14, 8.0);
      tot += om[s];
    }
    for (int l = 1; l < Mc; ++l) {
      double acc = 0.0;
      for (int s = 0; s < NSTEN; ++s)
        if (ok[s]) acc += (om[s] / tot) * wc[s][l][r];
      wchar[l][r] = acc;
    }
  }
  for (int v = 0; v < 4; ++v) {
    w[0 * 4 + v] = Qi[v];
    for (int l = 1; l < Mc; ++l) {
      double acc = 0.0;
      for (int r = 0; r < 4; ++r) acc += R[v * 4 + r] * wchar[l][r];
      w[l * 4 + v] = acc;
    }
  }
}

/* local time step of element i from its own and its edge neighbours' virtual
   data (eq. timestep, R9), in seconds */
static double local_dt(const oc_ctx* c, int64_t i, double cfl) {
  double best = HUGE_VAL;
  for (int e = -1; e < 3; ++e) {
    int64_t j = e < 0 ? i : c->nbr[i * 3 + e];
    if (j < 0) continue;
    double Xv[6], Qv[4];
    virtual_data(c, j, c->t[i], Xv, Qv);
    double area = tri_area(Xv);
    double per = 0.0;
    for (int k = 0; k < 3; ++k) {
      double dx = Xv[2 * ((k + 1) % 3)] - Xv[2 * k], dy = Xv[2 * ((k + 1) % 3) + 1] - Xv[2 * k + 1];
      per += sqrt(dx * dx + dy * dy);
    }
    double d = 4.0 * area / per;
    double u = Qv[1] / Qv[0], v = Qv[2] / Qv[0];
    double vel = sqrt(u * u + v * v);
    if (e < 0) /* an element on a moving wall counts the wall's speed (R16) */
      for (int k = 0; k < 3; ++k)
        if (c->edge_bc[c->elem_edge[i * 3 + k]] == 2) vel = fmax(vel, c->wall_speed);
    double lam = vel + sqrt(c->cfg.gamma * pressure(c, Qv) / Qv[0]);
    double dtj = cfl * d / lam;
    if (dtj < best) best = dtj;
  }
  return best;
}

/* ------------------------------------------------------------------------
 * local space-time Galerkin predictor (eqs. PDECG, pdef, Ktau, CGfinal,
 * ODEmesh, Vdof, newVertPos; R6)
 * ------------------------------------------------------------------------ */

static void predictor(const oc_ctx* c, const double* X, double dtsec, const double* w0, double* qh) {
  int Mc = c->Mc, Nt = c->Nt, Nst = c->Nst, nu = c->nu;
  double xh[MAXNST][2], x0[MAXMC][2];
  for (int s = 0; s < Mc; ++s) {
    x0[s][0] = X[0] + (X[2] - X[0]) * c->lat[s][0] + (X[4] - X[0]) * c->lat[s][1];
    x0[s][1] = X[1] + (X[3] - X[1]) * c->lat[s][0] + (X[5] - X[1]) * c->lat[s][1];
  }
  for (int t = 0; t < Nt; ++t)
    for (int s = 0; s < Mc; ++s) {
      for (int v = 0; v < 4; ++v) qh[(t * Mc + s) * 4 + v] = w0[s * 4 + v];
      xh[t * Mc + s][0] = x0[s][0];
      xh[t * Mc + s][1] = x0[s][1];
    }
  if (dtsec == 0.0) return;
  /* nodal differentiation matrices of the spatial Lagrange basis */
  double Dxi[MAXMC][MAXMC], Deta[MAXMC][MAXMC];
  for (int s = 0; s < Mc; ++s)
    for (int r = 0; r < Mc; ++r) {
      double dx = 0.0, de = 0.0;
      for (int a = 0; a < Mc; ++a) {
        int p = c->mono[a][0], q = c->mono[a][1];
        if (p > 0) dx += c->vinv[a][r] * p * ipow(c->lat[s][0], p - 1) * ipow(c->lat[s][1], q);
        if (q > 0) de += c->vinv[a][r] * q * ipow(c->lat[s][0], p) * ipow(c->lat[s][1], q - 1);
      }
      Dxi[s][r] = dx;
      Deta[s][r] = de;
    }
  for (int it = 0; it < c->nit; ++it) {
    double P[MAXNST][4], V[MAXNST][2];
    for (int t = 0; t < Nt; ++t) {
      double f[MAXMC][4], g[MAXMC][4];
      for (int s = 0; s < Mc; ++s) euler_flux(c, qh + (t * Mc + s) * 4, f[s], g[s]);
      for (int s = 0; s < Mc; ++s) {
        int l = t * Mc + s;
        double Qx[4] = {0}, Qe[4] = {0}, fx[4] = {0}, fe[4] = {0}, gx[4] = {0}, ge[4] = {0};
        double xx = 0, xe = 0, yx = 0, ye = 0;
        for (int r = 0; r < Mc; ++r) {
          for (int v = 0; v < 4; ++v) {
            Qx[v] += Dxi[s][r] * qh[(t * Mc + r) * 4 + v];
            Qe[v] += Deta[s][r] * qh[(t * Mc + r) * 4 + v];
            fx[v] += Dxi[s][r] * f[r][v];
            fe[v] += Deta[s][r] * f[r][v];
            gx[v] += Dxi[s][r] * g[r][v];
            ge[v] += Deta[s][r] * g[r][v];
          }
          xx += Dxi[s][r] * xh[t * Mc + r][0];
          xe += Deta[s][r] * xh[t * Mc + r][0];
          yx += Dxi[s][r] * xh[t * Mc + r][1];
          ye += Deta[s][r] * xh[t * Mc + r][1];
        }
        double xt = 0.0, yt = 0.0;
        for (int u = 0; u < Nt; ++u) {
          xt += c->Dtau[t][u] * xh[u * Mc + s][0];
          yt += c->Dtau[t][u] * xh[u * Mc + s][1];
        }
        xt /= dtsec;
        yt /= dtsec;
        /* inverse of the space-time Jacobian, eq. Jac */
        double det = xx * ye - xe * yx;
        double xix = ye / det, xiy = -xe / det, etx = -yx / det, ety = xx / det;
        double xit = -(xix * xt + xiy * yt), ett = -(etx * xt + ety * yt);
        for (int v = 0; v < 4; ++v)
          P[l][v] = -(Qx[v] * xit + Qe[v] * ett + fx[v] * xix + fe[v] * etx + gx[v] * xiy + ge[v] * ety);
        const double* q = qh + l * 4;
        V[l][0] = c->cfg.mesh_velocity == 1 ? 0.0 : q[1] / q[0];
        V[l][1] = c->cfg.mesh_velocity == 1 ? 0.0 : q[2] / q[0];
      }
    }
    /* K_tau qhat = dt M P with the tau=0 dofs known (eq. CGfinal), and the
       same for the vertex coordinates with V (eq. newVertPos) */
    double rhs[MAXNST * 6];
    for (int k = 0; k < nu; ++k) {
      int tk = 1 + k / Mc, sk = k % Mc;
      for (int v = 0; v < 6; ++v) {
        double acc = 0.0;
        for (int l = 0; l < Nst; ++l) {
          int tl = l / Mc, sl = l % Mc;
          double mkl = c->Ms[sk][sl] * c->Mt[tk][tl];
          double val = v < 4 ? P[l][v] : V[l][v - 4];
          acc += dtsec * mkl * val;
        }
        for (int sl = 0; sl < Mc; ++sl) {
          double kkl = c->Ms[sk][sl] * c->Kt[tk][0];
          double known = v < 4 ? qh[sl * 4 + v] : xh[sl][v - 4];
          acc -= kkl * known;
        }
        rhs[v * nu + k] = acc;
      }
    }
    for (int v = 0; v < 6; ++v) lu_solve(c->Kuu, c->piv, nu, rhs + v * nu);
    for (int k = 0; k < nu; ++k) {
      int l = Mc + k;
      for (int v = 0; v < 4; ++v) qh[l * 4 + v] = rhs[v * nu + k];
      xh[l][0] = rhs[4 * nu + k];
      xh[l][1] = rhs[5 * nu + k];
    }
  }
}

/* WENO polynomial at the lattice nodes, then the predictor of element i */
/* R11 positivity safeguards (not in the paper).  (a) If the WENO polynomial
   has a density or pressure below 1e-8 of the cell's own value at a lattice
   node, its non-constant part is scaled by the largest theta in [0,1] that
   keeps every node above that floor (the scaling of Zhang and Shu, 2010; for
   the pressure, which is concave in the conserved variables, theta comes from
   the chord bound p(Q + theta (w - Q)) >= (1 - theta) p(Q) + theta p(w)).
   (b) If the predictor ends with a non-positive density or pressure at a
   space-time node, the element keeps w_h at every time slice instead. */
static int physical(const oc_ctx* c, const double* q) { return q[0] > 0.0 && pressure(c, q) > 0.0; }
static void nodal_predictor(const oc_ctx* c, int64_t i, const double* w0);

static void element_predictor(const oc_ctx* c, int64_t i, const double* w) {
  double w0[MAXMC * 4];
  for (int s = 0; s < c->Mc; ++s) {
    double psi[MAXMC];
    dubiner_eval(c, c->lat[s][0], c->lat[s][1], psi);
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
      for (int l = 0; l < c->Mc; ++l) acc += psi[l] * w[l * 4 + v];
      w0[s * 4 + v] = acc;
    }
  }
  const double* Qi = c->Q + 4 * i;
  const double rho_min = 1e-8 * Qi[0], p_i = pressure(c, Qi), p_min = 1e-8 * p_i;
  for (int pass = 0; pass < 2; ++pass) {  /* density first, then pressure */
    double theta = 1.0;
    for (int s = 0; s < c->Mc; ++s) {
      const double* ws = w0 + 4 * s;
      if (pass == 0 && ws[0] < rho_min) {
        double th = (Qi[0] - rho_min) / (Qi[0] - ws[0]);
        if (th < theta) theta = th;
      }
      if (pass == 1) {
        double ps = pressure(c, ws);
        if (ps < p_min) {
          double th = (p_i - p_min) / (p_i - ps);
          if (th < theta) theta = th;
        }
      }
    }
    if (theta < 1.0)
      for (int s = 0; s < c->Mc; ++s)
        for (int v = 0; v < 4; ++v) w0[s * 4 + v] = Qi[v] + theta * (w0[s * 4 + v] - Qi[v]);
  }
  nodal_predictor(c, i, w0);
}

/* the predictor of element i over its step dt[i] from the nodal values w0 of
   its (scaled) WENO polynomial, with safeguard (b) */
static void nodal_predictor(const oc_ctx* c, int64_t i, const double* w0) {
  double* qh = c->qhat + (size_t)i * c->Nst * 4;
  predictor(c, c->X + 6 * i, (double)c->dt[i] * c->tick, w0, qh);
  int ok = 1;
  for (int l = 0; l < c->Nst && ok; ++l) ok = physical(c, qh + 4 * l);
  if (!ok)
    for (int t = 0; t < c->Nt; ++t)
      for (int s = 0; s < c->Mc; ++s)
        for (int v = 0; v < 4; ++v) qh[(t * c->Mc + s) * 4 + v] = w0[s * 4 + v];
}

/* ------------------------------------------------------------------------
 * phase B for a list of elements: reconstruction, dt, predictor
 * ------------------------------------------------------------------------ */

static int phase_b(oc_ctx* c, const int64_t* list, int64_t n) {
  double* W = (double*)malloc(sizeof(double) * (n > 0 ? n : 1) * c->Mc * 4);
  int64_t gmin = INT64_MAX;
  int rc = OC_OK;
  for (int64_t q = 0; q < n; ++q) {
    int64_t i = list[q];
    OC_PHASE(OC_PH_RECON);
    reconstruct(c, i, W + q * c->Mc * 4);
    OC_PHASE(OC_PH_DT);
    int64_t ticks = 0;
    const int start = c->t[i] < c->Tsw;  /* global-step start-up (R16) */
    if (c->t[i] < c->Ts) {
      double dts = local_dt(c, i, start ? c->cfg.cfl_start : c->cfg.cfl);
      if (!(dts > 0.0)) {
        rc = fail(c, OC_NONPHYSICAL, "element %lld: non-positive time step", (long long)i);
        break;
      }
      double r = floor(dts / c->tick);
      int64_t end = start ? c->Tsw : c->T;
      if (end > c->Ts) end = c->Ts;
      ticks = r > (double)(end - c->t[i]) ? end - c->t[i] : (int64_t)r;
      if (ticks < 1) ticks = 1;
    }
    if (c->sched_mode != 0) {
      if (c->count[i] >= c->sched_k) {
        rc = fail(c, OC_STATE, "element %lld: update %lld is beyond the schedule log", (long long)i,
                  (long long)c->count[i]);
        break;
      }
      int64_t* slot = c->sched_log + i * c->sched_k + c->count[i];
      if (c->sched_mode == 1) *slot = ticks;
      else ticks = *slot;
    }
    c->dt[i] = ticks;
    if (ticks > 0 && ticks < gmin && (c->cfg.gts || start)) gmin = ticks;
  }
  if (rc == OC_OK && gmin != INT64_MAX)
    for (int64_t q = 0; q < n; ++q)
      if (c->dt[list[q]] > 0 && (c->cfg.gts || c->t[list[q]] < c->Tsw)) c->dt[list[q]] = gmin;
  OC_PHASE(OC_PH_PRED);
  if (rc == OC_OK)
    for (int64_t q = 0; q < n; ++q) element_predictor(c, list[q], W + q * c->Mc * 4);
  OC_PHASE(OC_PH_OTHER);
  free(W);
  return rc;
}

/* ------------------------------------------------------------------------
 * public entry points
 * ------------------------------------------------------------------------ */

int oc_create(const oc_config* cfg, oc_ctx** out) {
  if (!cfg || !out || cfg->order_M < 1 || cfg->order_M > MAXM || !(cfg->t_end > 0) || cfg->time_quantum_log2 < 1 ||
      cfg->time_quantum_log2 > 50 || !(cfg->cfl > 0) || !(cfg->gamma > 1) || cfg->flux < 0 || cfg->flux > 1 ||
      (cfg->t_switch > 0.0 && !(cfg->cfl_start > 0)))
    return OC_INVALID;
  oc_ctx* c = (oc_ctx*)calloc(1, sizeof(oc_ctx));
  c->cfg = *cfg;
  c->M = cfg->order_M;
  c->Mc = (c->M + 1) * (c->M + 2) / 2;
  c->Nt = c->M + 1;
  c->Nst = c->Mc * c->Nt;
  c->ne = 2 * c->Mc;
  c->nit = cfg->predictor_iters > 0 ? cfg->predictor_iters : c->M + 1;
  c->T = (int64_t)1 << cfg->time_quantum_log2;
  c->Ts = c->T;
  c->tick = ldexp(cfg->t_end, -cfg->time_quantum_log2);
  c->wall_speed = sqrt(cfg->wall_u * cfg->wall_u + cfg->wall_v * cfg->wall_v);
  c->Tsw = 0;
  if (cfg->t_switch > 0.0) {
    double r = floor(cfg->t_switch / c->tick);
    c->Tsw = r >= (double)c->T ? c->T : (int64_t)r;
  }
  if (build_tables(c)) {
    free(c);
    return OC_INVALID;
  }
  *out = c;
  return OC_OK;
}

static void free_mesh(oc_ctx* c) {
  void* ptrs[] = {c->tri, c->bc, c->shift, c->edge_nodes, c->edge_elem, c->edge_loc, c->edge_bc, c->elem_edge,
                  c->nbr, c->nbr_shift, c->v2e_ptr, c->v2e, c->v2e_loc, c->node_type, c->node_n, c->sten,
                  c->sten_shift, c->sten_ok, c->sw_ptr, c->sw, c->Q, c->QM, c->HM, c->X, c->qhat, c->t,
                  c->dt, c->count, c->nX, c->nt, c->xy0};
  for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; ++k) free(ptrs[k]);
  c->tri = NULL; c->bc = NULL; c->shift = NULL; c->edge_nodes = NULL; c->edge_elem = NULL;
  c->edge_loc = NULL; c->edge_bc = NULL; c->elem_edge = NULL; c->nbr = NULL; c->nbr_shift = NULL;
  c->v2e_ptr = NULL; c->v2e = NULL; c->v2e_loc = NULL; c->node_type = NULL; c->node_n = NULL;
  c->sten = NULL; c->sten_shift = NULL; c->sten_ok = NULL; c->sw_ptr = NULL; c->sw = NULL;
  c->Q = NULL; c->QM = NULL; c->HM = NULL; c->X = NULL; c->qhat = NULL; c->t = NULL;
  c->dt = NULL; c->count = NULL; c->nX = NULL; c->nt = NULL; c->xy0 = NULL;
  free(c->sched_log);
  c->sched_log = NULL;
  c->sched_mode = 0;
  c->sched_k = 0;
  c->have_state = 0;
}

void oc_destroy(oc_ctx* c) {
  if (!c) return;
  free_mesh(c);
  free(c->Kuu);
  free(c->piv);
  free(c);
}

const char* oc_last_error(const oc_ctx* c) { return c ? c->err : "null context"; }

int oc_load_mesh(oc_ctx* c, int64_t n_nodes, const double* xy, int64_t n_tris, const int32_t* tri, const int8_t* bc,
                 const int8_t* shift, const double* period) {
  if (!c || n_nodes < 3 || n_tris < 1 || !xy || !tri || !bc) return OC_INVALID;
  if ((shift == NULL) != (period == NULL)) return fail(c, OC_INVALID, "shift and period go together");
  free_mesh(c);
  c->nn = n_nodes;
  c->ne_ = n_tris;
  for (int64_t q = 0; q < 3 * n_tris; ++q) {
    if (tri[q] < 0 || tri[q] >= n_nodes) return fail(c, OC_BAD_MESH, "node index out of range");
    if (bc[q] < -1 || bc[q] > 3) return fail(c, OC_BAD_MESH, "boundary tag out of range");
  }
  c->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * n_tris);
  memcpy(c->tri, tri, sizeof(int32_t) * 3 * n_tris);
  c->bc = (int8_t*)malloc(3 * n_tris);
  memcpy(c->bc, bc, 3 * n_tris);
  c->periodic = period != NULL;
  if (c->periodic) {
    c->shift = (int8_t*)malloc(6 * n_tris);
    memcpy(c->shift, shift, 6 * n_tris);
    c->period[0] = period[0];
    c->period[1] = period[1];
    if (!(period[0] >= 0.0 && period[1] >= 0.0 && period[0] + period[1] > 0.0))
      return fail(c, OC_INVALID, "period components must be >= 0, one of them positive");
  }
  int rc = build_mesh(c, xy);
  if (rc) return rc;
  c->Q = (double*)calloc(4 * n_tris, sizeof(double));
  c->QM = (double*)calloc(4 * n_tris, sizeof(double));
  c->HM = (double*)calloc(3 * n_tris, sizeof(double));
  c->X = (double*)calloc(6 * n_tris, sizeof(double));
  c->qhat = (double*)calloc((size_t)c->Nst * 4 * n_tris, sizeof(double));
  c->t = (int64_t*)calloc(n_tris, sizeof(int64_t));
  c->dt = (int64_t*)calloc(n_tris, sizeof(int64_t));
  c->count = (int64_t*)calloc(n_tris, sizeof(int64_t));
  c->nX = (double*)malloc(sizeof(double) * 2 * n_nodes);
  memcpy(c->nX, xy, sizeof(double) * 2 * n_nodes);
  c->xy0 = (double*)malloc(sizeof(double) * 2 * n_nodes);
  memcpy(c->xy0, xy, sizeof(double) * 2 * n_nodes);
  c->nt = (int64_t*)calloc(n_nodes, sizeof(int64_t));
  return OC_OK;
}

/* pre-processing phase (Sec. 2.6): cell averages at t=0, first WENO without
   virtual data, local time steps, predictor; node times 0 */
static int load_state(oc_ctx* c, const double* Q, const double* xy) {
  if (!c || !c->tri || !Q) return OC_INVALID;
  int64_t ne = c->ne_;
  memcpy(c->Q, Q, sizeof(double) * 4 * ne);
  memcpy(c->nX, xy ? xy : c->xy0, sizeof(double) * 2 * c->nn);
  for (int64_t i = 0; i < ne; ++i) {
    if (!(Q[4 * i] > 0.0) || !(pressure(c, Q + 4 * i) > 0.0))
      return fail(c, OC_NONPHYSICAL, "initial state of element %lld is not physical", (long long)i);
    for (int v = 0; v < 4; ++v) c->QM[4 * i + v] = 0.0;
    for (int v = 0; v < 3; ++v) c->HM[3 * i + v] = 0.0;
    c->t[i] = 0;
    c->count[i] = 0;
    for (int k = 0; k < 3; ++k) corner(c, i, k, c->nX, c->X + 6 * i + 2 * k);
  }
  for (int64_t n = 0; n < c->nn; ++n) c->nt[n] = 0;
  c->Ts = c->T;
  int64_t* all = (int64_t*)malloc(sizeof(int64_t) * ne);
  for (int64_t i = 0; i < ne; ++i) all[i] = i;
  int rc = phase_b(c, all, ne);
  free(all);
  c->gcl_max = 0.0;
  c->gcl_checked = 0.0;
  c->have_state = rc == OC_OK;
  return rc;
}

int oc_load_state(oc_ctx* c, const double* Q) { return load_state(c, Q, NULL); }

/* initial state on moved node positions; the mesh pre-processing (stencils,
   total stencils, wall normals) stays that of oc_load_mesh */
int oc_load_state_xy(oc_ctx* c, const double* Q, const double* xy) {
  if (!xy) return OC_INVALID;
  return load_state(c, Q, xy);
}

int oc_schedule(oc_ctx* c, int mode, int64_t k) {
  if (!c || !c->tri || mode < 0 || mode > 2) return OC_INVALID;
  if (mode != 0 && (c->cfg.gts || c->Tsw > 0))
    return fail(c, OC_INVALID, "the schedule log is for local time stepping");
  if (mode == 1) {
    if (k < 1) return OC_INVALID;
    free(c->sched_log);
    c->sched_log = (int64_t*)calloc((size_t)c->ne_ * k, sizeof(int64_t));
    c->sched_k = k;
  } else if (mode == 2 && !c->sched_log) {
    return fail(c, OC_STATE, "no recorded schedule to replay");
  }
  c->sched_mode = mode;
  return OC_OK;
}

int oc_get_schedule(const oc_ctx* c, int64_t* out) {
  if (!c || !c->sched_log || !out) return OC_INVALID;
  memcpy(out, c->sched_log, sizeof(int64_t) * c->ne_ * c->sched_k);
  return OC_OK;
}

int oc_set_schedule(oc_ctx* c, int64_t k, const int64_t* log) {
  if (!c || !c->tri || k < 1 || !log) return OC_INVALID;
  if (c->cfg.gts || c->Tsw > 0) return fail(c, OC_INVALID, "the schedule log is for local time stepping");
  free(c->sched_log);
  c->sched_log = (int64_t*)malloc(sizeof(int64_t) * (size_t)c->ne_ * (size_t)k);
  if (!c->sched_log) return fail(c, OC_INVALID, "out of memory");
  memcpy(c->sched_log, log, sizeof(int64_t) * (size_t)c->ne_ * (size_t)k);
  c->sched_k = k;
  return OC_OK;
}

/* one cycle of the LTS algorithm under the Jacobi reading R2 (Sec. 2.6) */
int oc_sweep(oc_ctx* c, int64_t* n_updated) {
  if (!c || !c->have_state) return OC_STATE;
  int64_t ne = c->ne_, nn = c->nn, T = c->Ts;
  int Mc = c->Mc, Nt = c->Nt, Nst = c->Nst;
  /* update criterion on the total stencil (eq. WENOupdate) */
  char* ready = (char*)calloc(ne, 1);
  int64_t nready = 0, unfinished = 0;
  for (int64_t i = 0; i < ne; ++i) {
    if (c->t[i] >= T) continue;
    ++unfinished;
    int64_t tn = c->t[i] + c->dt[i];
    int ok = 1;
    for (int64_t p = c->sw_ptr[i]; p < c->sw_ptr[i + 1] && ok; ++p) {
      int32_t j = c->sw[p];
      if (c->t[j] > tn || tn > c->t[j] + c->dt[j]) ok = 0;
    }
    if (ok) {
      ready[i] = 1;
      ++nready;
    }
  }
  if (n_updated) *n_updated = nready;
  if (nready == 0) {
    free(ready);
    if (unfinished) return fail(c, OC_DEADLOCK, "no element satisfies the update criterion");
    return OC_OK;
  }
  /* nodes of ready elements move to the common future time (Sec. 2.4) */
  char* moved = (char*)calloc(nn, 1);
  int64_t* tnew = (int64_t*)malloc(sizeof(int64_t) * nn);
  double* Xnew = (double*)malloc(sizeof(double) * 2 * nn);
  memcpy(Xnew, c->nX, sizeof(double) * 2 * nn);
  memcpy(tnew, c->nt, sizeof(int64_t) * nn);
  for (int64_t i = 0; i < ne; ++i)
    if (ready[i])
      for (int k = 0; k < 3; ++k) {
        int32_t n = c->tri[i * 3 + k];
        moved[n] = 1;
        tnew[n] = c->t[i] + c->dt[i];
      }
  OC_PHASE(OC_PH_NODES);
  /* node solver NS_cs: mass-weighted, time-integrated vertex velocities
     (eqs. eqnNScs, eqn.NScs.weights, dtau, NodesVel, newVertex; R7) */
  for (int64_t n = 0; n < nn; ++n) {
    if (!moved[n]) continue;
    double num[2] = {0.0, 0.0}, den = 0.0;
    for (int64_t p = c->v2e_ptr[n]; p < c->v2e_ptr[n + 1]; ++p) {
      int32_t j = c->v2e[p];
      int k = c->v2e_loc[p];
      double mu = c->Q[4 * j] * tri_area(c->X + 6 * j);
      double D[2] = {0.0, 0.0};
      if (c->dt[j] > 0) {
        double tau0 = (double)(c->nt[n] - c->t[j]) / (double)c->dt[j];
        double tau1 = (double)(tnew[n] - c->t[j]) / (double)c->dt[j];
        double I[2];
        vertex_velocity_integral(c, c->qhat + (size_t)j * Nst * 4, k, tau0, tau1, I);
        double dtj = (double)c->dt[j] * c->tick;
        D[0] = dtj * I[0];
        D[1] = dtj * I[1];
      }
      num[0] += mu * D[0];
      num[1] += mu * D[1];
      den += mu;
    }
    double D[2] = {num[0] / den, num[1] / den};
    if (c->node_type[n] == 1) {
      double dn = D[0] * c->node_n[2 * n] + D[1] * c->node_n[2 * n + 1];
      D[0] -= dn * c->node_n[2 * n];
      D[1] -= dn * c->node_n[2 * n + 1];
    } else if (c->node_type[n] == 2) {
      D[0] = D[1] = 0.0;
    } else if (c->node_type[n] == 3) {
      double span = (double)(tnew[n] - c->nt[n]) * c->tick;
      D[0] = c->cfg.wall_u * span;
      D[1] = c->cfg.wall_v * span;
    }
    Xnew[2 * n] = c->nX[2 * n] + D[0];
    Xnew[2 * n + 1] = c->nX[2 * n + 1] + D[1];
  }
  OC_PHASE(OC_PH_FLUX);
  /* space-time edge and vertex fluxes through the surfaces swept by every
     edge with a moved endpoint (eqs. spacetimenodes, rusanov, STint; R8) */
  int64_t ned = c->nedges;
  double* G = (double*)calloc(4 * ned, sizeof(double));
  double* N = (double*)calloc(3 * ned, sizeof(double));
  char* active = (char*)calloc(ned, 1);
  static const double refv[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
  for (int64_t ed = 0; ed < ned; ++ed) {
    int32_t a = c->edge_nodes[2 * ed], b = c->edge_nodes[2 * ed + 1];
    if (!moved[a] && !moved[b]) continue;
    active[ed] = 1;
    int32_t L = c->edge_elem[2 * ed], R = c->edge_elem[2 * ed + 1];
    int le = c->edge_loc[2 * ed], lr = c->edge_loc[2 * ed + 1];
    /* corners in the left element's frame: (X_a^n,t_a^n), (X_b^n,t_b^n),
       (X_b^{n+1},t_b^{n+1}), (X_a^{n+1},t_a^{n+1}) */
    double P[4][3];
    double sa[2] = {0.0, 0.0}, sb[2] = {0.0, 0.0};
    if (c->periodic) {
      sa[0] = c->shift[(L * 3 + le) * 2] * c->period[0];
      sa[1] = c->shift[(L * 3 + le) * 2 + 1] * c->period[1];
      sb[0] = c->shift[(L * 3 + (le + 1) % 3) * 2] * c->period[0];
      sb[1] = c->shift[(L * 3 + (le + 1) % 3) * 2 + 1] * c->period[1];
    }
    P[0][0] = c->nX[2 * a] + sa[0]; P[0][1] = c->nX[2 * a + 1] + sa[1]; P[0][2] = (double)c->nt[a] * c->tick;
    P[1][0] = c->nX[2 * b] + sb[0]; P[1][1] = c->nX[2 * b + 1] + sb[1]; P[1][2] = (double)c->nt[b] * c->tick;
    P[2][0] = Xnew[2 * b] + sb[0]; P[2][1] = Xnew[2 * b + 1] + sb[1]; P[2][2] = (double)tnew[b] * c->tick;
    P[3][0] = Xnew[2 * a] + sa[0]; P[3][1] = Xnew[2 * a + 1] + sa[1]; P[3][2] = (double)tnew[a] * c->tick;
    double tk[4] = {(double)c->nt[a], (double)c->nt[b], (double)tnew[b], (double)tnew[a]};
    const double* qL = c->qhat + (size_t)L * Nst * 4;
    const double* qR = R >= 0 ? c->qhat + (size_t)R * Nst * 4 : NULL;
    for (int gx = 0; gx < Nt; ++gx)
      for (int gt = 0; gt < Nt; ++gt) {
        double chi = c->glx[gx], tau = c->glx[gt], wq = c->glw[gx] * c->glw[gt];
        double dchi[3], dtau[3], n[3];
        for (int d = 0; d < 3; ++d) {
          dchi[d] = (1.0 - tau) * (P[1][d] - P[0][d]) + tau * (P[2][d] - P[3][d]);
          dtau[d] = (1.0 - chi) * (P[3][d] - P[0][d]) + chi * (P[2][d] - P[1][d]);
        }
        n[0] = dchi[1] * dtau[2] - dchi[2] * dtau[1];
        n[1] = dchi[2] * dtau[0] - dchi[0] * dtau[2];
        n[2] = dchi[0] * dtau[1] - dchi[1] * dtau[0];
        double tt = (1 - chi) * (1 - tau) * tk[0] + chi * (1 - tau) * tk[1] + chi * tau * tk[2] + (1 - chi) * tau * tk[3];
        double qm[4], qp[4];
        double tauL = c->dt[L] > 0 ? (tt - (double)c->t[L]) / (double)c->dt[L] : 0.0;
        eval_qh(c, qL, refv[le][0] + chi * (refv[(le + 1) % 3][0] - refv[le][0]),
                refv[le][1] + chi * (refv[(le + 1) % 3][1] - refv[le][1]), tauL, qm);
        if (R >= 0) {
          double tauR = c->dt[R] > 0 ? (tt - (double)c->t[R]) / (double)c->dt[R] : 0.0;
          double cr = 1.0 - chi;
          eval_qh(c, qR, refv[lr][0] + cr * (refv[(lr + 1) % 3][0] - refv[lr][0]),
                  refv[lr][1] + cr * (refv[(lr + 1) % 3][1] - refv[lr][1]), tauR, qp);
        } else if (c->edge_bc[ed] == 1) {
          /* transmissive: the boundary element's sweep-start average (R15) */
          for (int v = 0; v < 4; ++v) qp[v] = c->Q[4 * L + v];
        } else if (c->edge_bc[ed] == 3) {
          /* the exact Kidder state at the quadrature point (R17) */
          double px = (1 - chi) * (1 - tau) * P[0][0] + chi * (1 - tau) * P[1][0] + chi * tau * P[2][0] + (1 - chi) * tau * P[3][0];
          double py = (1 - chi) * (1 - tau) * P[0][1] + chi * (1 - tau) * P[1][1] + chi * tau * P[2][1] + (1 - chi) * tau * P[3][1];
          kidder_state(c, px, py, tt * c->tick, qp);
        } else {
          boundary_state(c, c->edge_bc[ed], qm, n, qp);
        }
        double F[4];
        num_flux(c, qm, qp, n, F);
        for (int v = 0; v < 4; ++v) G[4 * ed + v] += wq * F[v];
        for (int d = 0; d < 3; ++d) N[3 * ed + d] += wq * n[d];
      }
  }
  OC_PHASE(OC_PH_UPDATE);
  /* finite volume update with memory variables (eqs. PDEfinal, Qm2, gcl) */
  int rc = OC_OK;
  double* Qold = (double*)malloc(sizeof(double) * 4 * ne);
  memcpy(Qold, c->Q, sizeof(double) * 4 * ne);
  for (int64_t i = 0; i < ne; ++i) {
    double outG[3][4], outN[3][3];
    int any = 0, act[3];
    for (int e = 0; e < 3; ++e) {
      int32_t ed = c->elem_edge[i * 3 + e];
      act[e] = active[ed];
      if (!act[e]) continue;
      any = 1;
      double sg = c->edge_elem[2 * ed] == i ? 1.0 : -1.0;
      for (int v = 0; v < 4; ++v) outG[e][v] = sg * G[4 * ed + v];
      for (int d = 0; d < 3; ++d) outN[e][d] = sg * N[3 * ed + d];
    }
    if (!any) continue;
    if (ready[i]) {
      double Xn[6];
      for (int k = 0; k < 3; ++k) corner(c, i, k, Xnew, Xn + 2 * k);
      double Aold = tri_area(c->X + 6 * i), Anew = tri_area(Xn);
      double acc[4];
      for (int v = 0; v < 4; ++v) {
        acc[v] = Aold * c->Q[4 * i + v];
        for (int e = 0; e < 3; ++e)
          if (act[e]) acc[v] -= outG[e][v];
        acc[v] += c->QM[4 * i + v];
        c->Q[4 * i + v] = acc[v] / Anew;
        c->QM[4 * i + v] = 0.0;
      }
      double res[3];
      for (int d = 0; d < 3; ++d) {
        res[d] = 0.0;
        for (int e = 0; e < 3; ++e)
          if (act[e]) res[d] += outN[e][d];
        res[d] -= c->HM[3 * i + d];
        c->HM[3 * i + d] = 0.0;
      }
      res[2] += Anew - Aold;
      for (int d = 0; d < 3; ++d)
        if (fabs(res[d]) / Aold > c->gcl_max) c->gcl_max = fabs(res[d]) / Aold;
      c->gcl_checked += 1.0;
      memcpy(c->X + 6 * i, Xn, sizeof(double) * 6);
      c->t[i] += c->dt[i];
      c->count[i] += 1;
      if (!(c->Q[4 * i] > 0.0) || !(pressure(c, c->Q + 4 * i) > 0.0) || !(Anew > 0.0))
        if (rc == OC_OK) rc = fail(c, OC_NONPHYSICAL, "element %lld is non-physical after its update", (long long)i);
    } else {
      for (int e = 0; e < 3; ++e) {
        if (!act[e]) continue;
        for (int v = 0; v < 4; ++v) c->QM[4 * i + v] -= outG[e][v];
        for (int d = 0; d < 3; ++d) c->HM[3 * i + d] -= outN[e][d];
      }
    }
  }
  free(Qold);
  OC_PHASE(OC_PH_OTHER);
  memcpy(c->nX, Xnew, sizeof(double) * 2 * nn);
  memcpy(c->nt, tnew, sizeof(int64_t) * nn);
  if (rc == OC_OK) {
    int64_t* list = (int64_t*)malloc(sizeof(int64_t) * nready);
    int64_t q = 0;
    for (int64_t i = 0; i < ne; ++i)
      if (ready[i]) list[q++] = i;
    rc = phase_b(c, list, nready);
    free(list);
  }
  free(ready);
  free(moved);
  free(tnew);
  free(Xnew);
  free(G);
  free(N);
  free(active);
  if (rc != OC_OK) c->have_state = 0;
  (void)Mc;
  return rc;
}

/* Run sweeps until every element reached the sync time t (reading R18: t is
   t_end or a whole number of ticks, not behind any element's time) or
   max_sweeps sweeps ran.  Moving the sync time back cuts every step that
   crosses it back to it and re-solves that element's predictor over the
   shorter step from its own tau = 0 dofs (the scaled WENO values); moving
   it forward gives each element stopped at the old sync time its phase B
   (reconstruction, step, predictor) at that time. */
int oc_advance_to(oc_ctx* c, double t, int64_t max_sweeps, int64_t* sweeps_done, int64_t* updates_done) {
  if (!c || !c->have_state) return OC_STATE;
  int64_t ne = c->ne_, Tn = c->T;
  if (t < c->cfg.t_end) {
    double r = t / c->tick;
    if (!(r >= 0.0) || r != floor(r)) return fail(c, OC_INVALID, "the sync time is not a whole number of ticks");
    Tn = (int64_t)r;
  }
  for (int64_t i = 0; i < ne; ++i)
    if (c->t[i] > Tn) return fail(c, OC_INVALID, "element %lld is beyond the sync time", (long long)i);
  if (Tn != c->Ts && c->sched_mode != 0) return fail(c, OC_INVALID, "a sync time before t_end with a frozen schedule");
  int64_t* list = (int64_t*)malloc(sizeof(int64_t) * (ne > 0 ? ne : 1));
  int64_t n = 0;
  int rc = OC_OK;
  if (Tn < c->Ts) {
    for (int64_t i = 0; i < ne; ++i)
      if (c->t[i] < Tn && c->t[i] + c->dt[i] > Tn) {
        c->dt[i] = Tn - c->t[i];
        double w0[MAXMC * 4];
        memcpy(w0, c->qhat + (size_t)i * c->Nst * 4, sizeof(double) * c->Mc * 4);
        nodal_predictor(c, i, w0);
      }
    c->Ts = Tn;
  } else if (Tn > c->Ts) {
    for (int64_t i = 0; i < ne; ++i)
      if (c->t[i] == c->Ts) list[n++] = i;
    c->Ts = Tn;
    rc = phase_b(c, list, n);
  }
  free(list);
  if (rc != OC_OK) {
    c->have_state = 0;
    return rc;
  }
  int64_t sweeps = 0, updates = 0;
  while (sweeps < max_sweeps) {
    int64_t u = 0;
    rc = oc_sweep(c, &u);
    if (rc != OC_OK) return rc;
    if (u == 0) break;
    updates += u;
    ++sweeps;
  }
  if (sweeps_done) *sweeps_done = sweeps;
  if (updates_done) *updates_done = updates;
  return OC_OK;
}

int oc_get_elem(const oc_ctx* c, double* Q, double* QM, double* HM, int64_t* t, int64_t* dt, double* X,
                int64_t* count, double* qhat) {
  if (!c || !c->tri) return OC_INVALID;
  int64_t ne = c->ne_;
  if (Q) memcpy(Q, c->Q, sizeof(double) * 4 * ne);
  if (QM) memcpy(QM, c->QM, sizeof(double) * 4 * ne);
  if (HM) memcpy(HM, c->HM, sizeof(double) * 3 * ne);
  if (t) memcpy(t, c->t, sizeof(int64_t) * ne);
  if (dt) memcpy(dt, c->dt, sizeof(int64_t) * ne);
  if (X) memcpy(X, c->X, sizeof(double) * 6 * ne);
  if (count) memcpy(count, c->count, sizeof(int64_t) * ne);
  if (qhat) memcpy(qhat, c->qhat, sizeof(double) * c->Nst * 4 * ne);
  return OC_OK;
}

int oc_set_elem(oc_ctx* c, const double* Q, const double* QM, const double* HM, const int64_t* t, const int64_t* dt,
                const double* X, const int64_t* count, const double* qhat) {
  if (!c || !c->tri || !Q || !QM || !HM || !t || !dt || !X || !count || !qhat) return OC_INVALID;
  int64_t ne = c->ne_;
  memcpy(c->Q, Q, sizeof(double) * 4 * ne);
  memcpy(c->QM, QM, sizeof(double) * 4 * ne);
  memcpy(c->HM, HM, sizeof(double) * 3 * ne);
  memcpy(c->t, t, sizeof(int64_t) * ne);
  memcpy(c->dt, dt, sizeof(int64_t) * ne);
  memcpy(c->X, X, sizeof(double) * 6 * ne);
  memcpy(c->count, count, sizeof(int64_t) * ne);
  memcpy(c->qhat, qhat, sizeof(double) * c->Nst * 4 * ne);
  c->have_state = 1;
  return OC_OK;
}

int oc_get_nodes(const oc_ctx* c, double* X, int64_t* t) {
  if (!c || !c->tri) return OC_INVALID;
  if (X) memcpy(X, c->nX, sizeof(double) * 2 * c->nn);
  if (t) memcpy(t, c->nt, sizeof(int64_t) * c->nn);
  return OC_OK;
}

int oc_set_nodes(oc_ctx* c, const double* X, const int64_t* t) {
  if (!c || !c->tri || !X || !t) return OC_INVALID;
  memcpy(c->nX, X, sizeof(double) * 2 * c->nn);
  memcpy(c->nt, t, sizeof(int64_t) * c->nn);
  return OC_OK;
}

int64_t oc_n_st(const oc_ctx* c) { return c ? c->Nst : 0; }
int64_t oc_n_edges(const oc_ctx* c) { return c ? c->nedges : 0; }

int oc_diag(const oc_ctx* c, double* out) {
  if (!c || !out) return OC_INVALID;
  out[0] = c->gcl_max;
  out[1] = c->gcl_checked;
  return OC_OK;
}

int oc_get_stencils(const oc_ctx* c, int64_t i, int32_t* members, int32_t* sw, int cap) {
  if (!c || !c->tri || i < 0 || i >= c->ne_) return OC_INVALID;
  if (members) memcpy(members, c->sten + i * NSTEN * c->ne, sizeof(int32_t) * NSTEN * c->ne);
  int64_t n = c->sw_ptr[i + 1] - c->sw_ptr[i];
  if (sw)
    for (int64_t q = 0; q < n && q < cap; ++q) sw[q] = c->sw[c->sw_ptr[i] + q];
  return (int)n;
}

int oc_reconstruct_eval(oc_ctx* c, int64_t i, int64_t npts, const double* xy, double* out) {
  if (!c || !c->have_state || i < 0 || i >= c->ne_) return OC_INVALID;
  double w[MAXMC * 4];
  reconstruct(c, i, w);
  for (int64_t p = 0; p < npts; ++p) {
    double xi, eta, psi[MAXMC];
    to_reference(c->X + 6 * i, xy[2 * p], xy[2 * p + 1], &xi, &eta);
    dubiner_eval(c, xi, eta, psi);
    for (int v = 0; v < 4; ++v) {
      double acc = 0.0;
      for (int l = 0; l < c->Mc; ++l) acc += psi[l] * w[l * 4 + v];
      out[4 * p + v] = acc;
    }
  }
  return OC_OK;
}

int oc_predict_debug(oc_ctx* c, const double* X6, double dt_sec, const double* w_nodal, double* qhat_out) {
  if (!c || !X6 || !w_nodal || !qhat_out) return OC_INVALID;
  predictor(c, X6, dt_sec, w_nodal, qhat_out);
  return OC_OK;
}

int oc_flux_debug(const oc_ctx* c, const double* qL, const double* qR, const double* n3, int bc, double* out) {
  if (!c) return OC_INVALID;
  double qp[4];
  if (qR)
    memcpy(qp, qR, sizeof qp);
  else
    boundary_state(c, bc, qL, n3, qp);
  num_flux(c, qL, qp, n3, out);
  return OC_OK;
}

int oc_eval_qh(const oc_ctx* c, const double* qhat, int64_t npts, const double* pts, double* out) {
  if (!c) return OC_INVALID;
  for (int64_t p = 0; p < npts; ++p) eval_qh(c, qhat, pts[3 * p], pts[3 * p + 1], pts[3 * p + 2], out + 4 * p);
  return OC_OK;
}

int oc_table(const oc_ctx* c, int what, int64_t npts, const double* pts, double* out) {
  if (!c) return OC_INVALID;
  int Mc = c->Mc, Nt = c->Nt;
  switch (what) {
    case 0:
      for (int64_t p = 0; p < npts; ++p) dubiner_eval(c, pts[2 * p], pts[2 * p + 1], out + p * Mc);
      return OC_OK;
    case 1:
      for (int l = 0; l < Mc; ++l)
        for (int m = 0; m < Mc; ++m) out[l * Mc + m] = c->Sigma[l][m];
      return OC_OK;
    case 2:
      for (int t = 0; t < Nt; ++t) out[t] = c->tau[t];
      return OC_OK;
    case 3:
      for (int k = 0; k < Nt; ++k)
        for (int l = 0; l < Nt; ++l) out[k * Nt + l] = c->Kt[k][l];
      return OC_OK;
    case 4:
      for (int k = 0; k < Nt; ++k)
        for (int l = 0; l < Nt; ++l) out[k * Nt + l] = c->Mt[k][l];
      return OC_OK;
    case 5:
      for (int s = 0; s < Mc; ++s) {
        out[2 * s] = c->lat[s][0];
        out[2 * s + 1] = c->lat[s][1];
      }
      return OC_OK;
    case 6:
      if (npts < 1 || npts > 8) return OC_INVALID;
      gauss_legendre01((int)npts, out, out + npts);
      return OC_OK;
    case 7:
      for (int64_t p = 0; p < npts; ++p) lagrange_eval(c, pts[2 * p], pts[2 * p + 1], out + p * Mc);
      return OC_OK;
    default:
      return OC_INVALID;
  }
}
