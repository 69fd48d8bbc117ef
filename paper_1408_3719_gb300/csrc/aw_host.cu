// Host side of the GB300 ALE ADER-WENO LTS library: reference tables, mesh
// pre-processing (edges, Voronoi sets, stencils, symmetric total stencils),
// device memory, the sweep driver and the C ABI of include/aleweno.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/aleweno.h"
#include "aw_internal.h"

using namespace aw;

struct aw_ctx {
  aw_config cfg{};
  Tab tab{};
  Dev d{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = -1;           // current device at aw_create: every entry point runs there
  int nsm = 0;
  bool have_mesh = false, have_state = false, failed = false;
  bool moving_wall = false;  // the mesh has a moving slip wall or a Kidder boundary (tags 2, 3)
  std::vector<void*> allocs;
  Counters* hcnt = nullptr;  // pinned mirror of the device counters
  bool prof = false;         // per-kernel CUDA-event timing of sweeps
  cudaGraphExec_t prof_graph = nullptr;  // the sweep with an event before and after every kernel
  cudaEvent_t prof_ev[kNumKernels + 1] = {};
  // side stream of the sweep graph: the node solver runs beside the edge
  // marking (they read the moved-node list and write disjoint arrays)
  cudaStream_t side = nullptr;
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  double prof_ms[kNumKernels] = {0};
  long long prof_sweeps = 0;
  long long ne = 0, nn = 0, ned = 0, sw_total = 0, u_total = 0;
  std::vector<double> xy0;
  double* d_corner0 = nullptr;  // element corners at t = 0
  std::vector<double> etick_h, ntick_h;  // seconds per tick of each element / node
  cudaGraphExec_t graph_exec = nullptr;  // one captured sweep
  Tiles tiles;                           // tile shapes of the sweep kernels
  std::vector<int> tri_h;                // host copies for aw_load_state_xy
  std::vector<double> cshift_h;
  bool fresh = false;                    // a state was loaded and no sweep has run since
  bool batch = false;                    // loaded by aw_load_batch (ticks differ per instance)
  long long t_sync = 0;                  // the sync time in ticks (a copy of the device's)
  // frozen schedule (record / replay of the dt ticks)
  long long* d_sched = nullptr;
  // checkpointed forward run and its adjoint
  struct Snap {
    double *Q, *QM, *HM, *X, *qhat, *trace, *avgc, *vdisp, *nX;
    long long *t, *dt, *count, *nt;
    Counters* cnt;
  };
  std::vector<void*> adj_allocs;
  std::vector<Snap> ckpt;  // state before sweep m * adj_k
  Snap fin{};              // state after the run
  std::vector<Snap> slots; // sweep-start states of one segment
  Adj adjv{};
  double* d_gxy = nullptr;
  long long adj_n = 0, adj_k = 0;
  bool adj_ready = false;
  bool last_seg_kept = false;  // slots hold the last segment's sweep-start states
};

namespace {

int set_err(aw_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return set_err(c, AW_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// small exact polynomial algebra on the reference triangle (host only)
// ---------------------------------------------------------------------------
struct Poly {  // sum c[a][b] xi^a eta^b, total degree <= 8
  double c[9][9];
  Poly() { std::memset(c, 0, sizeof c); }
};

double factorial(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
double mono_integral(int a, int b) { return factorial(a) * factorial(b) / factorial(a + b + 2); }  // int over T_e

Poly mul(const Poly& p, const Poly& q) {
  Poly r;
  for (int a = 0; a < 9; ++a)
    for (int b = 0; a + b < 9; ++b)
      if (p.c[a][b] != 0)
        for (int e = 0; a + e < 9; ++e)
          for (int f = 0; a + b + e + f < 9; ++f) r.c[a + e][b + f] += p.c[a][b] * q.c[e][f];
  return r;
}
Poly deriv(const Poly& p, int da, int db) {
  Poly r;
  for (int a = da; a < 9; ++a)
    for (int b = db; b < 9; ++b) {
      double k = 1;
      for (int i = 0; i < da; ++i) k *= (a - i);
      for (int i = 0; i < db; ++i) k *= (b - i);
      r.c[a - da][b - db] += k * p.c[a][b];
    }
  return r;
}
double integral(const Poly& p) {
  double s = 0;
  for (int a = 0; a < 9; ++a)
    for (int b = 0; a + b < 9; ++b) s += p.c[a][b] * mono_integral(a, b);
  return s;
}
// (xi - 1/3)^a (eta - 1/3)^b expanded
Poly centred_monomial(int a, int b) {
  Poly r;
  for (int i = 0; i <= a; ++i)
    for (int j = 0; j <= b; ++j) {
      double ca = factorial(a) / (factorial(i) * factorial(a - i)) * std::pow(-1.0 / 3.0, a - i);
      double cb = factorial(b) / (factorial(j) * factorial(b - j)) * std::pow(-1.0 / 3.0, b - j);
      r.c[i][j] += ca * cb;
    }
  return r;
}

// Gauss-Jordan inverse with partial pivoting (n <= 16)
bool gj_inverse(std::vector<double> a, int n, std::vector<double>& inv) {
  inv.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[r * n + col]) > std::fabs(a[piv * n + col])) piv = r;
    if (a[piv * n + col] == 0.0) return false;
    for (int k = 0; k < n; ++k) {
      std::swap(a[col * n + k], a[piv * n + k]);
      std::swap(inv[col * n + k], inv[piv * n + k]);
    }
    double d = a[col * n + col];
    for (int k = 0; k < n; ++k) { a[col * n + k] /= d; inv[col * n + k] /= d; }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      double f = a[r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[col * n + k]; inv[r * n + k] -= f * inv[col * n + k]; }
    }
  }
  return true;
}

int build_tab(aw_ctx* c) {
  Tab& T = c->tab;
  const int M = c->cfg.order_M;
  T.M = M;
  T.Mc = (M + 1) * (M + 2) / 2;
  T.Nt = M + 1;
  T.Nst = T.Mc * T.Nt;
  T.NU = T.Mc - 1;
  T.gamma = c->cfg.gamma;
  T.cfl = c->cfg.cfl;
  T.T = 1LL << c->cfg.time_quantum_log2;
  T.tick = std::ldexp(c->cfg.t_end, -c->cfg.time_quantum_log2);
  T.eulerian = c->cfg.mesh_velocity == 1;
  T.gts = c->cfg.gts ? 1 : 0;
  T.nit = c->cfg.predictor_iters > 0 ? c->cfg.predictor_iters : M + 1;
  T.flux = c->cfg.flux;
  T.wall_u = c->cfg.wall_u;
  T.wall_v = c->cfg.wall_v;
  T.wall_speed = std::sqrt(c->cfg.wall_u * c->cfg.wall_u + c->cfg.wall_v * c->cfg.wall_v);
  T.cfl_start = c->cfg.cfl_start;
  for (int k = 0; k < 5; ++k) T.kidder[k] = c->cfg.kidder[k];
  T.Tsw = 0;
  if (c->cfg.t_switch > 0.0) {
    const double r = std::floor(c->cfg.t_switch / T.tick);
    T.Tsw = r >= (double)T.T ? T.T : (long long)r;
  }
  const int Mc = T.Mc, Nt = T.Nt;
  // lattice nodes: rows of constant eta, xi fastest
  int s = 0;
  for (int j = 0; j <= M; ++j)
    for (int i = 0; i <= M - j; ++i) { T.lat[s][0] = double(i) / M; T.lat[s][1] = double(j) / M; ++s; }
  T.vnode[0] = 0; T.vnode[1] = M; T.vnode[2] = Mc - 1;
  // Lagrange basis via a Vandermonde matrix in plain monomials (graded order)
  std::vector<std::pair<int, int>> ex;
  for (int dgr = 0; dgr <= M; ++dgr)
    for (int b = 0; b <= dgr; ++b) ex.push_back({dgr - b, b});
  std::vector<double> V(Mc * Mc), Vi;
  for (int r = 0; r < Mc; ++r)
    for (int k = 0; k < Mc; ++k) V[r * Mc + k] = std::pow(T.lat[r][0], ex[k].first) * std::pow(T.lat[r][1], ex[k].second);
  if (!gj_inverse(V, Mc, Vi)) return set_err(c, AW_ERR_INVALID_ARG, "singular lattice Vandermonde");
  std::vector<Poly> phi(Mc);
  for (int r = 0; r < Mc; ++r)
    for (int k = 0; k < Mc; ++k) phi[r].c[ex[k].first][ex[k].second] += Vi[k * Mc + r];
  auto peval = [](const Poly& p, double x, double y) {
    double v = 0;
    for (int a = 0; a < 9; ++a)
      for (int b = 0; a + b < 9; ++b)
        if (p.c[a][b] != 0) v += p.c[a][b] * std::pow(x, a) * std::pow(y, b);
    return v;
  };
  for (int r = 0; r < Mc; ++r) {
    Poly dx = deriv(phi[r], 1, 0), dy = deriv(phi[r], 0, 1);
    for (int q = 0; q < Mc; ++q) {
      T.Dxi[q][r] = peval(dx, T.lat[q][0], T.lat[q][1]);
      T.Deta[q][r] = peval(dy, T.lat[q][0], T.lat[q][1]);
    }
    T.wavg[r] = 2.0 * integral(phi[r]);
  }
  // Gauss-Lobatto times and the time Lagrange polynomials in monomial form
  double tau[kMaxNt];
  if (M == 1) { tau[0] = 0; tau[1] = 1; }
  else if (M == 2) { tau[0] = 0; tau[1] = 0.5; tau[2] = 1; }
  else { tau[0] = 0; tau[1] = 0.5 - std::sqrt(5.0) / 10.0; tau[2] = 0.5 + std::sqrt(5.0) / 10.0; tau[3] = 1; }
  std::vector<double> Vt(Nt * Nt), Vti;
  for (int t = 0; t < Nt; ++t)
    for (int p = 0; p < Nt; ++p) Vt[t * Nt + p] = std::pow(tau[t], p);
  if (!gj_inverse(Vt, Nt, Vti)) return set_err(c, AW_ERR_INVALID_ARG, "singular time Vandermonde");
  for (int p = 0; p < Nt; ++p)
    for (int t = 0; t < Nt; ++t) T.VtInv[p][t] = Vti[p * Nt + t];  // L_t(tau) = sum_p VtInv[p][t] tau^p
  // K_t = int L_k L_l', M_t = int L_k L_l on [0,1], exactly
  double Kt[kMaxNt][kMaxNt], Mt[kMaxNt][kMaxNt];
  for (int k = 0; k < Nt; ++k)
    for (int l = 0; l < Nt; ++l) {
      double kk = 0, mm = 0;
      for (int p = 0; p < Nt; ++p)
        for (int q = 0; q < Nt; ++q) {
          mm += T.VtInv[p][k] * T.VtInv[q][l] / (p + q + 1);
          if (q > 0) kk += T.VtInv[p][k] * q * T.VtInv[q][l] / (p + q);
        }
      Kt[k][l] = kk;
      Mt[k][l] = mm;
    }
  for (int t = 0; t < Nt; ++t)
    for (int u = 0; u < Nt; ++u) {
      double v = 0;
      for (int q = 1; q < Nt; ++q) v += T.VtInv[q][u] * q * std::pow(tau[t], q - 1);
      T.Dtau[t][u] = v;
    }
  // test functions of the tau > 0 nodes: K11 qhat_1 = dt M10.. P - K10 qhat_0, K10 = -K11 1
  std::vector<double> K11((Nt - 1) * (Nt - 1)), K11i;
  for (int a = 1; a < Nt; ++a)
    for (int b = 1; b < Nt; ++b) K11[(a - 1) * (Nt - 1) + (b - 1)] = Kt[a][b];
  if (!gj_inverse(K11, Nt - 1, K11i)) return set_err(c, AW_ERR_INVALID_ARG, "singular K11");
  for (int a = 0; a < Nt - 1; ++a)
    for (int u = 0; u < Nt; ++u) {
      double v = 0;
      for (int b = 0; b < Nt - 1; ++b) v += K11i[a * (Nt - 1) + b] * Mt[b + 1][u];
      T.B[a][u] = v;
    }
  // Gauss-Legendre points on [0,1] (closed forms)
  if (Nt == 2) {
    double h = 0.5 / std::sqrt(3.0);
    T.glx[0] = 0.5 - h; T.glx[1] = 0.5 + h; T.glw[0] = T.glw[1] = 0.5;
  } else if (Nt == 3) {
    double h = 0.5 * std::sqrt(0.6);
    T.glx[0] = 0.5 - h; T.glx[1] = 0.5; T.glx[2] = 0.5 + h;
    T.glw[0] = T.glw[2] = 5.0 / 18.0; T.glw[1] = 8.0 / 18.0;
  } else {
    double a = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(1.2)), b = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(1.2));
    double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    T.glx[0] = 0.5 - 0.5 * b; T.glx[1] = 0.5 - 0.5 * a; T.glx[2] = 0.5 + 0.5 * a; T.glx[3] = 0.5 + 0.5 * b;
    T.glw[0] = T.glw[3] = 0.5 * wb; T.glw[1] = T.glw[2] = 0.5 * wa;
  }
  const double rv[3][2] = {{0, 0}, {1, 0}, {0, 1}};
  for (int e = 0; e < 3; ++e)
    for (int g = 0; g < Nt; ++g) {
      double x = rv[e][0] + T.glx[g] * (rv[(e + 1) % 3][0] - rv[e][0]);
      double y = rv[e][1] + T.glx[g] * (rv[(e + 1) % 3][1] - rv[e][1]);
      for (int r = 0; r < Mc; ++r) T.Tr[e][g][r] = peval(phi[r], x, y);
    }
  // reconstruction basis: zero-mean centred monomials b_l, l = 1..Mc-1
  std::vector<Poly> bl;
  int l = 0;
  for (int dgr = 1; dgr <= M; ++dgr)
    for (int b = 0; b <= dgr; ++b) {
      T.mexp[l][0] = dgr - b;
      T.mexp[l][1] = b;
      Poly p = centred_monomial(dgr - b, b);
      T.mbar[l] = 2.0 * integral(p);
      bl.push_back(p);
      ++l;
    }
  for (int q = 0; q < Mc; ++q)
    for (int k = 0; k < T.NU; ++k) T.Bnod[q][k] = peval(bl[k], T.lat[q][0], T.lat[q][1]) - T.mbar[k];
  // smoothness matrix sigma = c^T S c, S_lm = sum_{1<=a+b<=M} int d^{ab} b_l d^{ab} b_m
  std::vector<double> S(T.NU * T.NU, 0.0);
  for (int i = 0; i < T.NU; ++i)
    for (int j = 0; j < T.NU; ++j) {
      double v = 0;
      for (int a = 0; a <= M; ++a)
        for (int b = 0; a + b <= M; ++b) {
          if (a + b == 0) continue;
          v += integral(mul(deriv(bl[i], a, b), deriv(bl[j], a, b)));
        }
      S[i * T.NU + j] = v;
    }
  // Cholesky S = U^T U (U upper)
  std::memset(T.SigU, 0, sizeof T.SigU);
  for (int j = 0; j < T.NU; ++j) {
    double d = S[j * T.NU + j];
    for (int k = 0; k < j; ++k) d -= T.SigU[k][j] * T.SigU[k][j];
    if (!(d > 0)) return set_err(c, AW_ERR_INVALID_ARG, "smoothness matrix not positive definite");
    T.SigU[j][j] = std::sqrt(d);
    for (int i = j + 1; i < T.NU; ++i) {
      double v = S[j * T.NU + i];
      for (int k = 0; k < j; ++k) v -= T.SigU[k][j] * T.SigU[k][i];
      T.SigU[j][i] = v / T.SigU[j][j];
    }
  }
  return AW_OK;
}

// ---------------------------------------------------------------------------
// mesh pre-processing on the host
// ---------------------------------------------------------------------------
struct HostMesh {
  int ne = 0, nn = 0, ned = 0;
  bool periodic = false;
  double period[2] = {0, 0};
  std::vector<int> tri;
  std::vector<signed char> bc, shift;
  std::vector<double> cshift, corner0, cen;
  std::vector<int> elem_edge, edge_nodes, edge_elem, nbr;
  std::vector<signed char> edge_loc, edge_bc, v2e_loc, node_type, sten_ok;
  std::vector<double> nbr_shift, node_n, u_shift;
  std::vector<int> v2e_ptr, v2e, sw_ptr, sw, u_ptr, u_elem, n2e_ptr, n2e;
  std::vector<unsigned char> sten;
};

// offset of element j's centroid seen from element i, nearest periodic image
inline void centroid_offset(const HostMesh& m, int i, int j, double& dx, double& dy, int& sx, int& sy) {
  dx = m.cen[2 * j] - m.cen[2 * i];
  dy = m.cen[2 * j + 1] - m.cen[2 * i + 1];
  sx = sy = 0;
  if (m.periodic) {  // a zero period component: not periodic in that direction
    if (m.period[0] > 0) sx = -(int)std::floor(dx / m.period[0] + 0.5);
    if (m.period[1] > 0) sy = -(int)std::floor(dy / m.period[1] + 0.5);
    dx = dx + sx * m.period[0];
    dy = dy + sy * m.period[1];
  }
}

int preprocess(aw_ctx* c, HostMesh& m, const double* xy, int ne_s, int M) {
  const int ne = m.ne, nn = m.nn;
  // corner offsets and t=0 corners
  m.cshift.assign(6 * (size_t)ne, 0.0);
  m.corner0.resize(6 * (size_t)ne);
  m.cen.resize(2 * (size_t)ne);
  for (int i = 0; i < ne; ++i) {
    for (int k = 0; k < 3; ++k) {
      if (m.periodic) {
        m.cshift[6 * i + 2 * k] = m.shift[6 * i + 2 * k] * m.period[0];
        m.cshift[6 * i + 2 * k + 1] = m.shift[6 * i + 2 * k + 1] * m.period[1];
      }
      int n = m.tri[3 * i + k];
      m.corner0[6 * i + 2 * k] = xy[2 * n] + m.cshift[6 * i + 2 * k];
      m.corner0[6 * i + 2 * k + 1] = xy[2 * n + 1] + m.cshift[6 * i + 2 * k + 1];
    }
    const double* X = &m.corner0[6 * i];
    double area2 = (X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0]);
    if (!(area2 > 0)) return set_err(c, AW_ERR_BAD_MESH, "element %d is not counter-clockwise", i);
    m.cen[2 * i] = (X[0] + X[2] + X[4]) / 3.0;
    m.cen[2 * i + 1] = (X[1] + X[3] + X[5]) / 3.0;
  }
  // node -> element CSR (ascending element index)
  m.v2e_ptr.assign(nn + 1, 0);
  for (int i = 0; i < ne; ++i)
    for (int k = 0; k < 3; ++k) m.v2e_ptr[m.tri[3 * i + k] + 1]++;
  std::partial_sum(m.v2e_ptr.begin(), m.v2e_ptr.end(), m.v2e_ptr.begin());
  m.v2e.resize(3 * (size_t)ne);
  m.v2e_loc.resize(3 * (size_t)ne);
  {
    std::vector<int> fill(m.v2e_ptr.begin(), m.v2e_ptr.end() - 1);
    for (int i = 0; i < ne; ++i)
      for (int k = 0; k < 3; ++k) {
        int p = fill[m.tri[3 * i + k]]++;
        m.v2e[p] = i;
        m.v2e_loc[p] = (signed char)k;
      }
  }
  // twins through a sorted list of directed edges
  struct DE { long long key; int elem, loc; };
  std::vector<DE> des(3 * (size_t)ne);
  for (int i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      long long a = m.tri[3 * i + e], b = m.tri[3 * i + (e + 1) % 3];
      des[3 * i + e] = {a * nn + b, i, e};
    }
  std::sort(des.begin(), des.end(), [](const DE& x, const DE& y) { return x.key < y.key || (x.key == y.key && x.elem < y.elem); });
  for (size_t q = 1; q < des.size(); ++q)
    if (des[q].key == des[q - 1].key) return set_err(c, AW_ERR_BAD_MESH, "repeated directed edge (non-manifold mesh)");
  m.nbr.assign(3 * (size_t)ne, -1);
  std::vector<signed char> nloc(3 * (size_t)ne, -1);
  for (int i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      long long a = m.tri[3 * i + e], b = m.tri[3 * i + (e + 1) % 3];
      long long key = b * nn + a;
      auto it = std::lower_bound(des.begin(), des.end(), key, [](const DE& x, long long k) { return x.key < k; });
      if (it != des.end() && it->key == key) {
        m.nbr[3 * i + e] = it->elem;
        nloc[3 * i + e] = (signed char)it->loc;
      } else if (m.bc[3 * i + e] < 0) {
        return set_err(c, AW_ERR_BAD_MESH, "boundary edge of element %d has no boundary tag", i);
      }
    }
  // canonical edges: element order, owner = the lower element index
  m.elem_edge.assign(3 * (size_t)ne, -1);
  m.edge_nodes.clear(); m.edge_elem.clear(); m.edge_loc.clear(); m.edge_bc.clear();
  int ned = 0;
  for (int i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      int j = m.nbr[3 * i + e];
      if (j >= 0 && j < i) { m.elem_edge[3 * i + e] = m.elem_edge[3 * j + nloc[3 * i + e]]; continue; }
      m.elem_edge[3 * i + e] = ned++;
      m.edge_nodes.push_back(m.tri[3 * i + e]);
      m.edge_nodes.push_back(m.tri[3 * i + (e + 1) % 3]);
      m.edge_elem.push_back(i);
      m.edge_elem.push_back(j);
      m.edge_loc.push_back((signed char)e);
      m.edge_loc.push_back(j >= 0 ? nloc[3 * i + e] : (signed char)-1);
      m.edge_bc.push_back(j >= 0 ? (signed char)-1 : m.bc[3 * i + e]);
    }
  m.ned = ned;
  // node -> incident edges
  m.n2e_ptr.assign(nn + 1, 0);
  for (int ed = 0; ed < ned; ++ed)
    for (int q = 0; q < 2; ++q) m.n2e_ptr[m.edge_nodes[2 * ed + q] + 1]++;
  std::partial_sum(m.n2e_ptr.begin(), m.n2e_ptr.end(), m.n2e_ptr.begin());
  m.n2e.resize(2 * (size_t)ned);
  {
    std::vector<int> fill(m.n2e_ptr.begin(), m.n2e_ptr.end() - 1);
    for (int ed = 0; ed < ned; ++ed)
      for (int q = 0; q < 2; ++q) m.n2e[fill[m.edge_nodes[2 * ed + q]]++] = ed;
  }
  // neighbour image offsets
  m.nbr_shift.assign(6 * (size_t)ne, 0.0);
  for (int i = 0; i < ne; ++i)
    for (int e = 0; e < 3; ++e) {
      int j = m.nbr[3 * i + e];
      if (j < 0) continue;
      double dx, dy;
      int sx, sy;
      centroid_offset(m, i, j, dx, dy, sx, sy);
      m.nbr_shift[6 * i + 2 * e] = sx * m.period[0];
      m.nbr_shift[6 * i + 2 * e + 1] = sy * m.period[1];
    }
  // slip-wall constraints of the nodes
  m.node_type.assign(nn, 0);
  m.node_n.assign(2 * (size_t)nn, 0.0);
  for (int ed = 0; ed < ned; ++ed) {
    if (m.edge_bc[ed] != 0) continue;
    int i = m.edge_elem[2 * ed], e = m.edge_loc[2 * ed];
    const double* X = &m.corner0[6 * i];
    double dx = X[2 * ((e + 1) % 3)] - X[2 * e], dy = X[2 * ((e + 1) % 3) + 1] - X[2 * e + 1];
    double len = std::sqrt(dx * dx + dy * dy);
    double n0 = dy / len, n1 = -dx / len;
    for (int q = 0; q < 2; ++q) {
      int nd = m.edge_nodes[2 * ed + q];
      if (m.node_type[nd] == 0) {
        m.node_type[nd] = 1; m.node_n[2 * nd] = n0; m.node_n[2 * nd + 1] = n1;
      } else if (m.node_type[nd] == 1) {
        if (std::fabs(m.node_n[2 * nd] * n1 - m.node_n[2 * nd + 1] * n0) > 1e-8) m.node_type[nd] = 2;
      }
    }
  }
  // nodes of moving walls move with the wall
  for (int ed = 0; ed < m.ned; ++ed)
    if (m.edge_bc[ed] == 2)
      for (int q = 0; q < 2; ++q) m.node_type[m.edge_nodes[2 * ed + q]] = 3;
  // stencils: candidates within vertex-neighbour layers, ordered by centroid distance then index
  m.sten.assign((size_t)ne * kNSten * ne_s, 0);
  m.sten_ok.assign((size_t)ne * kNSten, 0);
  m.u_ptr.assign(ne + 1, 0);
  m.u_elem.clear();
  m.u_shift.clear();
  std::vector<int> mark(ne, -1), layer, members;
  struct Cand { double d2; int j, sx, sy; };
  std::vector<Cand> cand;
  int stamp = 0;
  auto gather = [&](int i, int depth) {
    layer.clear();
    layer.push_back(i);
    mark[i] = ++stamp;
    size_t begin = 0;
    for (int dl = 0; dl < depth; ++dl) {
      size_t end = layer.size();
      for (size_t q = begin; q < end; ++q) {
        int e = layer[q];
        for (int k = 0; k < 3; ++k) {
          int nd = m.tri[3 * e + k];
          for (int p = m.v2e_ptr[nd]; p < m.v2e_ptr[nd + 1]; ++p) {
            int j = m.v2e[p];
            if (mark[j] != stamp) { mark[j] = stamp; layer.push_back(j); }
          }
        }
      }
      begin = end;
    }
    cand.clear();
    for (int j : layer) {
      Cand cd;
      double dx, dy;
      centroid_offset(m, i, j, dx, dy, cd.sx, cd.sy);
      cd.d2 = dx * dx + dy * dy;
      cd.j = j;
      cand.push_back(cd);
    }
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) { return a.d2 < b.d2 || (a.d2 == b.d2 && a.j < b.j); });
  };
  std::vector<int> sten_elem(kNSten * ne_s);
  std::vector<int> sten_sx(kNSten * ne_s), sten_sy(kNSten * ne_s);
  for (int i = 0; i < ne; ++i) {
    std::fill(sten_elem.begin(), sten_elem.end(), -1);
    gather(i, M + 1);
    if ((int)cand.size() < ne_s) return set_err(c, AW_ERR_BAD_MESH, "element %d: only %d candidates for the central stencil", i, (int)cand.size());
    for (int q = 0; q < ne_s; ++q) { sten_elem[q] = cand[q].j; sten_sx[q] = cand[q].sx; sten_sy[q] = cand[q].sy; }
    m.sten_ok[(size_t)i * kNSten] = 1;
    gather(i, M + 2);
    const double* X = &m.corner0[6 * i];
    double cx = m.cen[2 * i], cy = m.cen[2 * i + 1];
    for (int s = 1; s < kNSten; ++s) {
      int e = (s - 1) % 3;
      bool reverse = s >= 4;
      double ax = X[2 * e] - cx, ay = X[2 * e + 1] - cy;
      double bx = X[2 * ((e + 1) % 3)] - cx, by = X[2 * ((e + 1) % 3) + 1] - cy;
      int cntm = 0;
      sten_elem[s * ne_s + cntm] = i; sten_sx[s * ne_s] = 0; sten_sy[s * ne_s] = 0; ++cntm;
      for (size_t q = 0; q < cand.size() && cntm < ne_s; ++q) {
        if (cand[q].j == i) continue;
        double dx = m.cen[2 * cand[q].j] - cx + cand[q].sx * (m.periodic ? m.period[0] : 0.0);
        double dy = m.cen[2 * cand[q].j + 1] - cy + cand[q].sy * (m.periodic ? m.period[1] : 0.0);
        double al = dx * by - dy * bx;
        double be = ax * dy - ay * dx;
        bool in = reverse ? (al <= 0.0 && be <= 0.0) : (al >= 0.0 && be >= 0.0);
        if (!in) continue;
        sten_elem[s * ne_s + cntm] = cand[q].j;
        sten_sx[s * ne_s + cntm] = cand[q].sx;
        sten_sy[s * ne_s + cntm] = cand[q].sy;
        ++cntm;
      }
      if (cntm == ne_s) m.sten_ok[(size_t)i * kNSten + s] = 1;
      else for (int q = 0; q < ne_s; ++q) sten_elem[s * ne_s + q] = -1;
    }
    // unique member list (without i) and local indices
    members.clear();
    for (int q = 0; q < kNSten * ne_s; ++q)
      if (sten_elem[q] >= 0 && sten_elem[q] != i) members.push_back(sten_elem[q]);
    std::sort(members.begin(), members.end());
    members.erase(std::unique(members.begin(), members.end()), members.end());
    if (members.size() > 254) return set_err(c, AW_ERR_BAD_MESH, "element %d: stencil union too large", i);
    int base = (int)m.u_elem.size();
    for (int j : members) {
      m.u_elem.push_back(j);
      double dx, dy;
      int sx, sy;
      centroid_offset(m, i, j, dx, dy, sx, sy);
      m.u_shift.push_back(sx * m.period[0]);
      m.u_shift.push_back(sy * m.period[1]);
    }
    m.u_ptr[i + 1] = (int)m.u_elem.size();
    for (int q = 0; q < kNSten * ne_s; ++q) {
      int j = sten_elem[q];
      unsigned char loc = 0;
      if (j >= 0 && j != i) loc = (unsigned char)(1 + (std::lower_bound(members.begin(), members.end(), j) - members.begin()));
      m.sten[(size_t)i * kNSten * ne_s + q] = loc;
    }
    (void)base;
  }
  // total stencil: stencils + edge neighbours + Voronoi sets of the vertices, closed under symmetry
  std::vector<std::vector<int>> S(ne);
  for (int i = 0; i < ne; ++i) {
    auto& L = S[i];
    L.push_back(i);
    for (int p = m.u_ptr[i]; p < m.u_ptr[i + 1]; ++p) L.push_back(m.u_elem[p]);
    for (int e = 0; e < 3; ++e)
      if (m.nbr[3 * i + e] >= 0) L.push_back(m.nbr[3 * i + e]);
    for (int k = 0; k < 3; ++k) {
      int nd = m.tri[3 * i + k];
      for (int p = m.v2e_ptr[nd]; p < m.v2e_ptr[nd + 1]; ++p) L.push_back(m.v2e[p]);
    }
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
  }
  std::vector<std::vector<int>> Sx(S);
  for (int i = 0; i < ne; ++i)
    for (int j : S[i]) Sx[j].push_back(i);
  m.sw_ptr.assign(ne + 1, 0);
  m.sw.clear();
  for (int i = 0; i < ne; ++i) {
    auto& L = Sx[i];
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    m.sw.insert(m.sw.end(), L.begin(), L.end());
    m.sw_ptr[i + 1] = (int)m.sw.size();
  }
  return AW_OK;
}

template <class T>
int dalloc(aw_ctx* c, T** p, size_t n) {
  void* q = nullptr;
  if (n == 0) n = 1;
  CK(cudaMalloc(&q, n * sizeof(T)));
  c->allocs.push_back(q);
  *p = (T*)q;
  return AW_OK;
}

template <class T>
int dupload(aw_ctx* c, const T** out, const std::vector<T>& v) {
  T* p = nullptr;
  int rc = dalloc(c, &p, v.size());
  if (rc) return rc;
  if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  *out = p;
  return AW_OK;
}

// the captured sweeps become invalid when the tiles, the schedule mode or the
// mesh change
void drop_graphs(aw_ctx* c) {
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  if (c->prof_graph) {
    cudaGraphExecDestroy(c->prof_graph);
    c->prof_graph = nullptr;
  }
}

void free_all(aw_ctx* c) {
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
  for (void* p : c->adj_allocs) cudaFree(p);
  c->adj_allocs.clear();
  c->ckpt.clear();
  c->slots.clear();
  c->adjv = Adj{};
  c->d_gxy = nullptr;
  c->adj_ready = false;
  c->d_sched = nullptr;
  c->have_mesh = c->have_state = false;
  c->fresh = false;
}

// Counters and epoch stamps restart together (a stale stamp equal to a new
// epoch would mark an element or node as active).
int reset_sweep_state(aw_ctx* c) {
  const Dev& d = c->d;
  CK(cudaMemsetAsync(d.elem_ready, 0, c->ne * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.elem_touch, 0, c->ne * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.node_moved, 0, c->nn * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.edge_act, 0, c->ned * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.cand_stamp, 0, c->ne * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.cnt, 0, sizeof(Counters), c->stream));
  static const int one = 1;  // stamps are 0: the first sweep must be epoch 1
  CK(cudaMemcpyAsync(&d.cnt->epoch, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&d.cnt->t_sync, &c->t_sync, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return AW_OK;
}

// elements with t < t_sync, counted on the host from the device times
int count_unfinished(aw_ctx* c, long long* max_t) {
  std::vector<long long> th(c->ne);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(th.data(), c->d.t, c->ne * sizeof(long long), cudaMemcpyDeviceToHost));
  int unf = 0;
  long long mx = 0;
  for (long long v : th) {
    unf += v < c->t_sync;
    mx = std::max(mx, v);
  }
  if (max_t) *max_t = mx;
  CK(cudaMemcpy(&c->d.cnt->n_unfinished, &unf, sizeof(int), cudaMemcpyHostToDevice));
  return AW_OK;
}

int sync_counters(aw_ctx* c) {
  CK(cudaMemcpyAsync(c->hcnt, c->d.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return AW_OK;
}

int check_device_error(aw_ctx* c) {
  if (c->hcnt->err_code != 0) {
    c->failed = true;
    if (c->hcnt->err_code == AW_ERR_STATE)
      return set_err(c, AW_ERR_STATE,
                     "element %d: update beyond the recorded schedule, or a positivity safeguard acted in a "
                     "differentiated sweep", c->hcnt->err_elem);
    return set_err(c, c->hcnt->err_code, "element %d is non-physical after its update (rho, p or area <= 0)", c->hcnt->err_elem);
  }
  return AW_OK;
}

}  // namespace

// read-only access to a context for the allocation-free entry point
namespace aw {
bool ctx_view(aw_ctx* c, CtxView* v) {
  if (!c || !c->have_state || c->failed) return false;
  v->d = &c->d;
  v->T = c->t_sync;
  v->stream = c->stream;
  v->device = c->device;
  return true;
}
void ctx_error(aw_ctx* c, const char* msg) {
  if (c) c->err = msg;
}
}  // namespace aw

// ---------------------------------------------------------------------------
// snapshots of the sweep state for the checkpointed adjoint
// ---------------------------------------------------------------------------
namespace {

int adj_alloc(aw_ctx* c, void** p, size_t bytes) {
  if (cudaMalloc(p, bytes) != cudaSuccess)
    return set_err(c, AW_ERR_CUDA, "cudaMalloc of %zu bytes for the adjoint failed", bytes);
  c->adj_allocs.push_back(*p);
  return AW_OK;
}

int snap_alloc(aw_ctx* c, aw_ctx::Snap* s, std::vector<void*>* owner = nullptr) {
  const size_t ne = c->ne, nn = c->nn, Nt = c->tab.Nt;
  const size_t nd[9] = {4 * ne, 4 * ne, 4 * ne, 6 * ne, ne * c->tab.Nst * 4, ne * 3 * Nt * Nt * 4, ne * Nt * 4,
                        ne * 6 * Nt, 2 * nn};
  const size_t nl[4] = {ne, ne, ne, nn};
  size_t bytes = 0;
  auto pad = [](size_t b) { return (b + 255) & ~(size_t)255; };
  for (size_t k : nd) bytes += pad(k * sizeof(double));
  for (size_t k : nl) bytes += pad(k * sizeof(long long));
  bytes += pad(sizeof(Counters));
  void* base = nullptr;
  int rc;
  if (owner) {
    if (cudaMalloc(&base, bytes) != cudaSuccess) return set_err(c, AW_ERR_CUDA, "cudaMalloc of %zu bytes failed", bytes);
    owner->push_back(base);
  } else if ((rc = adj_alloc(c, &base, bytes))) {
    return rc;
  }
  char* p = (char*)base;
  double** dp[9] = {&s->Q, &s->QM, &s->HM, &s->X, &s->qhat, &s->trace, &s->avgc, &s->vdisp, &s->nX};
  for (int k = 0; k < 9; ++k) { *dp[k] = (double*)p; p += pad(nd[k] * sizeof(double)); }
  long long** lp[4] = {&s->t, &s->dt, &s->count, &s->nt};
  for (int k = 0; k < 4; ++k) { *lp[k] = (long long*)p; p += pad(nl[k] * sizeof(long long)); }
  s->cnt = (Counters*)p;
  return AW_OK;
}

// save = true: live -> snapshot; false: snapshot -> live (the per-sweep
// counters are then reset with the epoch still growing)
int snap_copy(aw_ctx* c, const aw_ctx::Snap& s, bool save) {
  const Dev& d = c->d;
  const size_t ne = c->ne, nn = c->nn, Nt = c->tab.Nt;
  struct { void* live; void* snap; size_t bytes; } arr[] = {
      {d.Q, s.Q, 4 * ne * sizeof(double)}, {d.QM, s.QM, 4 * ne * sizeof(double)},
      {d.HM, s.HM, 4 * ne * sizeof(double)}, {d.X, s.X, 6 * ne * sizeof(double)},
      {d.qhat, s.qhat, ne * c->tab.Nst * 4 * sizeof(double)}, {d.trace, s.trace, ne * 3 * Nt * Nt * 4 * sizeof(double)},
      {d.avgc, s.avgc, ne * Nt * 4 * sizeof(double)}, {d.vdisp, s.vdisp, ne * 6 * Nt * sizeof(double)},
      {d.nX, s.nX, 2 * nn * sizeof(double)}, {d.t, s.t, ne * sizeof(long long)}, {d.dt, s.dt, ne * sizeof(long long)},
      {d.count, s.count, ne * sizeof(long long)}, {d.nt, s.nt, nn * sizeof(long long)}};
  const void* src[13];
  void* dst[13];
  long long n8[13];
  int k = 0;
  for (auto& a : arr) {
    src[k] = save ? a.live : a.snap;
    dst[k] = save ? a.snap : a.live;
    n8[k] = (long long)(a.bytes / 8);
    ++k;
  }
  launch_multi_copy(src, dst, n8, k, c->nsm, c->stream);
  CK(cudaGetLastError());
  if (save) {
    CK(cudaMemcpyAsync(s.cnt, d.cnt, sizeof(Counters), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    launch_adj_reset(d, s.cnt, c->stream);
    CK(cudaGetLastError());
  }
  return AW_OK;
}

Dev snap_view(const aw_ctx* c, const aw_ctx::Snap& s) {
  Dev v = c->d;
  v.Q = s.Q; v.QM = s.QM; v.HM = s.HM; v.X = s.X; v.qhat = s.qhat; v.trace = s.trace; v.avgc = s.avgc;
  v.vdisp = s.vdisp; v.nX = s.nX; v.t = s.t; v.dt = s.dt; v.count = s.count; v.nt = s.nt;
  return v;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int aw_create(const aw_config* cfg, aw_ctx** out) {
  if (!cfg || !out) return AW_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->order_M < 1 || cfg->order_M > kMaxM || !(cfg->t_end > 0) || cfg->time_quantum_log2 < 1 ||
      cfg->time_quantum_log2 > 50 || !(cfg->cfl > 0) || !(cfg->gamma > 1) || cfg->mesh_velocity < 0 ||
      cfg->mesh_velocity > 1 || cfg->flux < 0 || cfg->flux > 1 || (cfg->t_switch > 0.0 && !(cfg->cfl_start > 0)))
    return AW_ERR_INVALID_ARG;
  aw_ctx* c = new aw_ctx();
  c->cfg = *cfg;
  int rc = build_tab(c);
  if (rc) { delete c; return rc; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    delete c;
    return AW_ERR_CUDA;
  }
  c->device = dev;
  if (cfg->cuda_stream) c->stream = (cudaStream_t)cfg->cuda_stream;
  else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return AW_ERR_CUDA; }
    c->own_stream = true;
  }
  if (cudaMallocHost(&c->hcnt, sizeof(Counters)) != cudaSuccess) { delete c; return AW_ERR_CUDA; }
  *out = c;
  return AW_OK;
}

void aw_destroy(aw_ctx* c) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_all(c);
  for (cudaEvent_t e : c->prof_ev)
    if (e) cudaEventDestroy(e);
  if (c->fork_ev) cudaEventDestroy(c->fork_ev);
  if (c->join_ev) cudaEventDestroy(c->join_ev);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->hcnt) cudaFreeHost(c->hcnt);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* aw_last_error(const aw_ctx* c) { return c ? c->err.c_str() : "null context"; }

// Shared by aw_load_mesh and aw_load_batch; etick (host, may be NULL for a
// uniform tick) gives each element's seconds per tick.
static int load_common(aw_ctx* c, int64_t n_nodes, const double* xy, int64_t n_tris, const int32_t* tri,
                       const int8_t* bc, const int8_t* shift, const double* period, const double* etick) {
  if (!c) return AW_ERR_INVALID_ARG;
  if (n_nodes < 3 || n_tris < 1 || !xy || !tri || !bc || n_nodes > (1LL << 30) || n_tris > (1LL << 29))
    return set_err(c, AW_ERR_INVALID_ARG, "bad mesh sizes or null arrays");
  if ((shift == nullptr) != (period == nullptr)) return set_err(c, AW_ERR_INVALID_ARG, "shift and period go together");
  free_all(c);
  c->t_sync = c->tab.T;
  HostMesh m;
  m.ne = (int)n_tris;
  m.nn = (int)n_nodes;
  std::vector<double> hxy(2 * n_nodes);
  m.tri.resize(3 * n_tris);
  m.bc.resize(3 * n_tris);
  // accept host or device pointers
  if (cudaMemcpy(hxy.data(), xy, hxy.size() * sizeof(double), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(m.tri.data(), tri, m.tri.size() * sizeof(int), cudaMemcpyDefault) != cudaSuccess ||
      cudaMemcpy(m.bc.data(), bc, m.bc.size(), cudaMemcpyDefault) != cudaSuccess)
    return set_err(c, AW_ERR_CUDA, "copying the mesh arrays failed");
  for (int v : m.tri)
    if (v < 0 || v >= n_nodes) return set_err(c, AW_ERR_BAD_MESH, "node index out of range");
  c->moving_wall = false;
  for (signed char b : m.bc) {
    if (b < -1 || b > 3) return set_err(c, AW_ERR_BAD_MESH, "boundary tag out of range");
    c->moving_wall |= b == 2 || b == 3;
  }
  if (period) {
    m.periodic = true;
    m.shift.resize(6 * n_tris);
    if (cudaMemcpy(m.shift.data(), shift, m.shift.size(), cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(m.period, period, 2 * sizeof(double), cudaMemcpyDefault) != cudaSuccess)
      return set_err(c, AW_ERR_CUDA, "copying the periodic data failed");
    if (!(m.period[0] >= 0 && m.period[1] >= 0 && m.period[0] + m.period[1] > 0))
      return set_err(c, AW_ERR_INVALID_ARG, "period components must be >= 0, one of them positive");
  } else {
    m.shift.assign(6 * n_tris, 0);
  }
  const int ne_s = 2 * c->tab.Mc;
  int rc = preprocess(c, m, hxy.data(), ne_s, c->tab.M);
  if (rc) return rc;
  Dev& d = c->d;
  d = Dev{};
  d.ne = m.ne; d.nn = m.nn; d.ned = m.ned; d.periodic = m.periodic;
  d.period[0] = m.period[0]; d.period[1] = m.period[1];
  const Tab& T = c->tab;
  if ((rc = dupload(c, &d.tri, m.tri)) || (rc = dupload(c, &d.cshift, m.cshift)) || (rc = dupload(c, &d.elem_edge, m.elem_edge)) ||
      (rc = dupload(c, &d.edge_nodes, m.edge_nodes)) || (rc = dupload(c, &d.edge_elem, m.edge_elem)) ||
      (rc = dupload(c, &d.edge_loc, m.edge_loc)) || (rc = dupload(c, &d.edge_bc, m.edge_bc)) || (rc = dupload(c, &d.nbr, m.nbr)) ||
      (rc = dupload(c, &d.nbr_shift, m.nbr_shift)) || (rc = dupload(c, &d.v2e_ptr, m.v2e_ptr)) || (rc = dupload(c, &d.v2e, m.v2e)) ||
      (rc = dupload(c, &d.v2e_loc, m.v2e_loc)) || (rc = dupload(c, &d.n2e_ptr, m.n2e_ptr)) ||
      (rc = dupload(c, &d.n2e, m.n2e)) || (rc = dupload(c, &d.node_type, m.node_type)) ||
      (rc = dupload(c, &d.node_n, m.node_n)) || (rc = dupload(c, &d.sw_ptr, m.sw_ptr)) || (rc = dupload(c, &d.sw, m.sw)) ||
      (rc = dupload(c, &d.u_ptr, m.u_ptr)) || (rc = dupload(c, &d.u_elem, m.u_elem)) || (rc = dupload(c, &d.u_shift, m.u_shift)) ||
      (rc = dupload(c, &d.sten, m.sten)) || (rc = dupload(c, &d.sten_ok, m.sten_ok)))
    return rc;
  c->etick_h.assign(m.ne, T.tick);
  if (etick) std::copy(etick, etick + m.ne, c->etick_h.begin());
  c->ntick_h.assign(m.nn, T.tick);
  for (int i = 0; i < m.ne; ++i)
    for (int k = 0; k < 3; ++k) c->ntick_h[m.tri[3 * i + k]] = c->etick_h[i];
  if ((rc = dupload(c, &d.etick, c->etick_h))) return rc;
  const size_t ne = m.ne, nn = m.nn, ned = m.ned;
  if ((rc = dalloc(c, &d.Q, 4 * ne)) || (rc = dalloc(c, &d.QM, 4 * ne)) || (rc = dalloc(c, &d.HM, 4 * ne)) ||
      (rc = dalloc(c, &d.t, ne)) || (rc = dalloc(c, &d.dt, ne)) || (rc = dalloc(c, &d.X, 6 * ne)) ||
      (rc = dalloc(c, &d.count, ne)) || (rc = dalloc(c, &d.qhat, ne * T.Nst * 4)) ||
      (rc = dalloc(c, &d.trace, ne * 3 * T.Nt * T.Nt * 4)) || (rc = dalloc(c, &d.avgc, ne * T.Nt * 4)) ||
      (rc = dalloc(c, &d.vdisp, ne * 3 * 2 * T.Nt)) || (rc = dalloc(c, &d.nX, 2 * nn)) || (rc = dalloc(c, &d.nt, nn)) ||
      (rc = dalloc(c, &d.nXn, 2 * nn)) || (rc = dalloc(c, &d.ntn, nn)) || (rc = dalloc(c, &d.elem_ready, ne)) ||
      (rc = dalloc(c, &d.elem_touch, ne)) || (rc = dalloc(c, &d.node_moved, nn)) || (rc = dalloc(c, &d.edge_act, ned)) ||
      (rc = dalloc(c, &d.ready_list, ne)) || (rc = dalloc(c, &d.moved_list, nn)) || (rc = dalloc(c, &d.active_list, ned)) ||
      (rc = dalloc(c, &d.touch_list, ne)) || (rc = dalloc(c, &d.cand_stamp, ne)) ||
      (rc = dalloc(c, &d.cand_list, 2 * ne)) || (rc = dalloc(c, &d.G, 4 * ned)) || (rc = dalloc(c, &d.N, 4 * ned)) ||
      (rc = dalloc(c, &d.w0, ne * T.Mc * 4)) || (rc = dalloc(c, &d.cnt, 1)))
    return rc;
  CK(cudaMemsetAsync(d.elem_ready, 0, ne * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.elem_touch, 0, ne * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.node_moved, 0, nn * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.edge_act, 0, ned * sizeof(int), c->stream));
  CK(cudaMemsetAsync(d.cnt, 0, sizeof(Counters), c->stream));
  CK(cudaMemcpyAsync(d.nX, hxy.data(), 2 * nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->xy0 = hxy;
  c->tri_h = m.tri;
  c->cshift_h = m.cshift;
  c->ne = m.ne; c->nn = m.nn; c->ned = m.ned; c->sw_total = (long long)m.sw.size();
  c->u_total = (long long)m.u_elem.size();
  c->have_mesh = true;
  c->have_state = false;
  c->failed = false;
  if ((rc = dalloc(c, &c->d_corner0, 6 * ne))) return rc;
  CK(cudaMemcpy(c->d_corner0, m.corner0.data(), 6 * ne * sizeof(double), cudaMemcpyHostToDevice));
  return AW_OK;
}

int aw_load_mesh(aw_ctx* c, int64_t n_nodes, const double* xy, int64_t n_tris, const int32_t* tri,
                 const int8_t* bc, const int8_t* shift, const double* period) {
  DeviceGuard dg_(c ? c->device : -1);
  if (c) c->batch = false;
  return load_common(c, n_nodes, xy, n_tris, tri, bc, shift, period, nullptr);
}

int aw_load_batch(aw_ctx* c, int n_inst, const int64_t* node_offsets, const int64_t* tri_offsets,
                  const double* t_end, const double* xy, const int32_t* tri, const int8_t* bc) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (n_inst < 1 || !node_offsets || !tri_offsets || !t_end || !xy || !tri || !bc)
    return set_err(c, AW_ERR_INVALID_ARG, "aw_load_batch: null arrays or no instance");
  if (c->tab.Tsw > 0) return set_err(c, AW_ERR_INVALID_ARG, "aw_load_batch: no global-step start-up in a batch");
  std::vector<int64_t> no(node_offsets, node_offsets + n_inst + 1), to(tri_offsets, tri_offsets + n_inst + 1);
  if (no[0] != 0 || to[0] != 0) return set_err(c, AW_ERR_INVALID_ARG, "aw_load_batch: offsets must start at 0");
  for (int k = 0; k < n_inst; ++k)
    if (no[k + 1] <= no[k] || to[k + 1] <= to[k] || !(t_end[k] > 0))
      return set_err(c, AW_ERR_INVALID_ARG, "aw_load_batch: instance %d is empty or has t_end <= 0", k);
  const int64_t nn = no[n_inst], ne = to[n_inst];
  std::vector<int32_t> gtri(3 * ne);
  if (cudaMemcpy(gtri.data(), tri, gtri.size() * sizeof(int32_t), cudaMemcpyDefault) != cudaSuccess)
    return set_err(c, AW_ERR_CUDA, "aw_load_batch: copying tri failed");
  std::vector<double> et(ne);
  for (int k = 0; k < n_inst; ++k) {
    const double tick = std::ldexp(t_end[k], -c->cfg.time_quantum_log2);
    for (int64_t i = to[k]; i < to[k + 1]; ++i) {
      et[i] = tick;
      for (int q = 0; q < 3; ++q) {
        const int64_t v = gtri[3 * i + q];
        if (v < 0 || v >= no[k + 1] - no[k])
          return set_err(c, AW_ERR_BAD_MESH, "aw_load_batch: instance %d has a node index out of range", k);
        gtri[3 * i + q] = (int32_t)(v + no[k]);
      }
    }
  }
  const int rc = load_common(c, nn, xy, ne, gtri.data(), bc, nullptr, nullptr, et.data());
  c->batch = rc == AW_OK;
  return rc;
}

static int load_state_impl(aw_ctx* c, const double* Q, const double* xy) {
  if (!c || !Q) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  const size_t ne = c->ne, nn = c->nn;
  std::vector<double> hQ(4 * ne);
  CK(cudaMemcpy(hQ.data(), Q, hQ.size() * sizeof(double), cudaMemcpyDefault));
  const double g = c->tab.gamma;
  for (size_t i = 0; i < ne; ++i) {
    const double* q = &hQ[4 * i];
    double p = (g - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
    if (!(q[0] > 0) || !(p > 0)) return set_err(c, AW_ERR_NONPHYSICAL, "initial state of element %zu is not physical", i);
  }
  std::vector<double> hxy, corners;
  if (xy) {
    hxy.resize(2 * nn);
    CK(cudaMemcpy(hxy.data(), xy, hxy.size() * sizeof(double), cudaMemcpyDefault));
    corners.resize(6 * ne);
    for (size_t i = 0; i < ne; ++i)
      for (int k = 0; k < 3; ++k) {
        const int n = c->tri_h[3 * i + k];
        corners[6 * i + 2 * k] = hxy[2 * n] + c->cshift_h[6 * i + 2 * k];
        corners[6 * i + 2 * k + 1] = hxy[2 * n + 1] + c->cshift_h[6 * i + 2 * k + 1];
      }
    for (size_t i = 0; i < ne; ++i) {
      const double* X = &corners[6 * i];
      if (!(0.5 * ((X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0])) > 0))
        return set_err(c, AW_ERR_BAD_MESH, "element %zu is not counter-clockwise at the given node positions", i);
    }
  }
  Dev& d = c->d;
  CK(cudaMemcpyAsync(d.Q, hQ.data(), 4 * ne * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(d.QM, 0, 4 * ne * sizeof(double), c->stream));
  CK(cudaMemsetAsync(d.HM, 0, 4 * ne * sizeof(double), c->stream));
  CK(cudaMemsetAsync(d.t, 0, ne * sizeof(long long), c->stream));
  CK(cudaMemsetAsync(d.count, 0, ne * sizeof(long long), c->stream));
  if (xy) {
    CK(cudaMemcpyAsync(d.X, corners.data(), 6 * ne * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(d.nX, hxy.data(), 2 * nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  } else {
    CK(cudaMemcpyAsync(d.X, c->d_corner0, 6 * ne * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(d.nX, c->xy0.data(), 2 * nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  CK(cudaMemsetAsync(d.nt, 0, nn * sizeof(long long), c->stream));
  c->t_sync = c->tab.T;
  int rc0 = reset_sweep_state(c);
  if (rc0) return rc0;
  {
    int unf = (int)ne;
    CK(cudaMemcpyAsync(&d.cnt->n_unfinished, &unf, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }

  launch_initial(c->tab, d, c->nsm, c->stream, c->tiles);
  CK(cudaGetLastError());
  int rc = sync_counters(c);
  if (rc) return rc;
  if ((rc = check_device_error(c))) return rc;
  c->have_state = true;
  c->failed = false;
  c->fresh = true;
  c->adj_ready = false;
  return AW_OK;
}

int aw_load_state(aw_ctx* c, const double* Q) {
  DeviceGuard dg_(c ? c->device : -1);
  return load_state_impl(c, Q, nullptr);
}

int aw_load_state_xy(aw_ctx* c, const double* Q, const double* xy) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !xy) return AW_ERR_INVALID_ARG;
  return load_state_impl(c, Q, xy);
}

static int do_sweeps(aw_ctx* c, int64_t n, int64_t* n_updated, bool wait) {
  if (!c->have_state || c->failed) return set_err(c, AW_ERR_STATE, "no valid state (load a state first)");
  if (n > 0) c->fresh = false;
  // A sweep is one CUDA-graph launch (captured once per mesh and tile shape).
  // With profiling it is a second graph with an event record between the
  // kernels: each profiled sweep waits for its last event and adds the
  // kernel times (the kernels run as in the plain graph).
  if (!c->prof && !c->graph_exec) {
    if (!c->side) {
      CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming));
    }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    launch_sweep(c->tab, c->d, c->nsm, c->stream, nullptr, c->tiles, c->side, c->fork_ev, c->join_ev);
    CK(cudaStreamEndCapture(c->stream, &g));
    CK(cudaGraphInstantiate(&c->graph_exec, g, 0));
    cudaGraphDestroy(g);
  }
  if (c->prof && !c->prof_graph) {
    for (cudaEvent_t& e : c->prof_ev)
      if (!e) CK(cudaEventCreate(&e));
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    launch_sweep(c->tab, c->d, c->nsm, c->stream, c->prof_ev, c->tiles);
    CK(cudaStreamEndCapture(c->stream, &g));
    CK(cudaGraphInstantiate(&c->prof_graph, g, 0));
    cudaGraphDestroy(g);
  }
  for (int64_t k = 0; k < n; ++k) {
    if (c->prof) {
      CK(cudaGraphLaunch(c->prof_graph, c->stream));
      CK(cudaEventSynchronize(c->prof_ev[kNumKernels]));
      for (int q = 0; q < kNumKernels; ++q) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, c->prof_ev[q], c->prof_ev[q + 1]));
        c->prof_ms[q] += ms;
      }
      c->prof_sweeps += 1;
    } else {
      CK(cudaGraphLaunch(c->graph_exec, c->stream));
    }
  }
  CK(cudaGetLastError());
  if (!wait) return AW_OK;
  int rc = sync_counters(c);
  if (rc) return rc;
  if ((rc = check_device_error(c))) return rc;
  if (n_updated) *n_updated = c->hcnt->last_ready;
  if (c->hcnt->last_ready == 0 && c->hcnt->n_unfinished > 0) {
    c->failed = true;
    return set_err(c, AW_ERR_DEADLOCK, "no element satisfies the update criterion (%d unfinished)", c->hcnt->n_unfinished);
  }
  return AW_OK;
}

int aw_lts_sweep(aw_ctx* c, int64_t* n_updated) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  return do_sweeps(c, 1, n_updated, true);
}

int aw_gts_step(aw_ctx* c, int64_t* n_updated) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->cfg.gts) return set_err(c, AW_ERR_INVALID_ARG, "aw_gts_step needs a context created with gts = 1");
  return do_sweeps(c, 1, n_updated, true);
}

// Reading R18: the run to a sync time t_s is the run whose final time is t_s.
// Moving the sync time back cuts the steps that cross it (predictors
// re-solved over the shorter steps); moving it forward gives the elements
// stopped at the old sync time their phase B there.
static int set_sync_time(aw_ctx* c, long long Tn) {
  if (Tn == c->t_sync) return AW_OK;
  if (c->d.sched_mode != 0)
    return set_err(c, AW_ERR_INVALID_ARG, "aw_advance_to: a sync time before t_end with a frozen schedule");
  long long max_t = 0;
  int rc = count_unfinished(c, &max_t);
  if (rc) return rc;
  if (max_t > Tn) return set_err(c, AW_ERR_INVALID_ARG, "aw_advance_to: an element is beyond the sync time");
  const long long Told = c->t_sync;
  c->t_sync = Tn;
  c->fresh = false;  // the adjoint starts from a state just loaded
  CK(cudaMemcpyAsync(&c->d.cnt->t_sync, &c->t_sync, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
  if (Tn < Told) launch_sync_cut(c->tab, c->d, c->nsm, c->stream, Tn, c->tiles);
  else launch_sync_resume(c->tab, c->d, c->nsm, c->stream, Told, c->tiles);
  CK(cudaGetLastError());
  if ((rc = count_unfinished(c, nullptr))) return rc;
  if ((rc = sync_counters(c))) return rc;
  return check_device_error(c);
}

int aw_advance_to(aw_ctx* c, double t, int64_t max_sweeps, int64_t* sweeps_done, int64_t* updates_done) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_state || c->failed) return set_err(c, AW_ERR_STATE, "no valid state (load a state first)");
  if (max_sweeps < 0) return set_err(c, AW_ERR_INVALID_ARG, "aw_advance_to: max_sweeps < 0");
  long long Tn = c->tab.T;
  if (t < c->cfg.t_end) {
    if (c->batch) return set_err(c, AW_ERR_INVALID_ARG, "aw_advance_to: a batch runs to its instances' t_end");
    const double r = t / c->tab.tick;
    if (!(r >= 0.0) || r != std::floor(r))
      return set_err(c, AW_ERR_INVALID_ARG, "aw_advance_to: t is not a whole number of ticks");
    Tn = (long long)r;
  }
  int rc = set_sync_time(c, Tn);
  if (rc) return rc;
  // sweeps go out in chunks between host checks; a sweep with an empty ready
  // set changes nothing, so overshooting the end of the run is harmless
  if ((rc = sync_counters(c))) return rc;
  const long long u0 = c->hcnt->updates, p0 = c->hcnt->productive;
  int64_t issued = 0, chunk = 8;
  while (issued < max_sweeps && c->hcnt->n_unfinished > 0) {
    const int64_t n = std::min<int64_t>(chunk, max_sweeps - issued);
    if ((rc = do_sweeps(c, n, nullptr, true))) return rc;
    issued += n;
    if (c->hcnt->n_unfinished == 0) break;
    if (c->hcnt->last_ready == 0) {
      c->failed = true;
      return set_err(c, AW_ERR_DEADLOCK, "no element satisfies the update criterion (%d unfinished)", c->hcnt->n_unfinished);
    }
    chunk = std::min<int64_t>(chunk * 2, 256);
  }
  if (sweeps_done) *sweeps_done = c->hcnt->productive - p0;
  if (updates_done) *updates_done = c->hcnt->updates - u0;
  return AW_OK;
}

int aw_enqueue_sweeps(aw_ctx* c, int64_t n) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || n < 0) return AW_ERR_INVALID_ARG;
  return do_sweeps(c, n, nullptr, false);
}

int aw_sync(aw_ctx* c, int64_t* updates_since) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  int rc = sync_counters(c);
  if (rc) return rc;
  if ((rc = check_device_error(c))) return rc;
  if (updates_since) *updates_since = c->hcnt->updates_since_sync;
  CK(cudaMemsetAsync(&c->d.cnt->updates_since_sync, 0, sizeof(long long), c->stream));
  return AW_OK;
}

int aw_get_state(aw_ctx* c, double* Q, double* t_elem) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  CK(cudaStreamSynchronize(c->stream));
  if (Q) CK(cudaMemcpy(Q, c->d.Q, 4 * c->ne * sizeof(double), cudaMemcpyDefault));
  if (t_elem) {
    std::vector<long long> t(c->ne);
    CK(cudaMemcpy(t.data(), c->d.t, c->ne * sizeof(long long), cudaMemcpyDeviceToHost));
    std::vector<double> td(c->ne);
    for (long long i = 0; i < c->ne; ++i) td[i] = (double)t[i] * c->etick_h[i];
    CK(cudaMemcpy(t_elem, td.data(), c->ne * sizeof(double), cudaMemcpyDefault));
  }
  return AW_OK;
}

int aw_get_nodes(aw_ctx* c, double* xy, double* t_node) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  CK(cudaStreamSynchronize(c->stream));
  if (xy) CK(cudaMemcpy(xy, c->d.nX, 2 * c->nn * sizeof(double), cudaMemcpyDefault));
  if (t_node) {
    std::vector<long long> t(c->nn);
    CK(cudaMemcpy(t.data(), c->d.nt, c->nn * sizeof(long long), cudaMemcpyDeviceToHost));
    std::vector<double> td(c->nn);
    for (long long i = 0; i < c->nn; ++i) td[i] = (double)t[i] * c->ntick_h[i];
    CK(cudaMemcpy(t_node, td.data(), c->nn * sizeof(double), cudaMemcpyDefault));
  }
  return AW_OK;
}

int aw_get_update_counts(aw_ctx* c, int64_t* per_elem, int64_t* total) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  int rc = sync_counters(c);
  if (rc) return rc;
  if (per_elem) CK(cudaMemcpy(per_elem, c->d.count, c->ne * sizeof(long long), cudaMemcpyDefault));
  if (total) *total = c->hcnt->updates;
  return AW_OK;
}

int aw_get_elem_arrays(aw_ctx* c, double* Q, double* QM, double* HM, int64_t* t, int64_t* dt, double* X,
                       int64_t* count, double* qhat) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  CK(cudaStreamSynchronize(c->stream));
  const size_t ne = c->ne;
  if (Q) CK(cudaMemcpy(Q, c->d.Q, 4 * ne * sizeof(double), cudaMemcpyDefault));
  if (QM) CK(cudaMemcpy(QM, c->d.QM, 4 * ne * sizeof(double), cudaMemcpyDefault));
  if (HM) CK(cudaMemcpy2D(HM, 3 * sizeof(double), c->d.HM, 4 * sizeof(double), 3 * sizeof(double), ne, cudaMemcpyDefault));
  if (t) CK(cudaMemcpy(t, c->d.t, ne * sizeof(long long), cudaMemcpyDefault));
  if (dt) CK(cudaMemcpy(dt, c->d.dt, ne * sizeof(long long), cudaMemcpyDefault));
  if (X) CK(cudaMemcpy(X, c->d.X, 6 * ne * sizeof(double), cudaMemcpyDefault));
  if (count) CK(cudaMemcpy(count, c->d.count, ne * sizeof(long long), cudaMemcpyDefault));
  if (qhat) CK(cudaMemcpy(qhat, c->d.qhat, ne * c->tab.Nst * 4 * sizeof(double), cudaMemcpyDefault));
  return AW_OK;
}

int aw_set_elem_arrays(aw_ctx* c, const double* Q, const double* QM, const double* HM, const int64_t* t,
                       const int64_t* dt, const double* X, const int64_t* count, const double* qhat) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !Q || !QM || !HM || !t || !dt || !X || !count || !qhat) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  const size_t ne = c->ne;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->d.Q, Q, 4 * ne * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.QM, QM, 4 * ne * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemset(c->d.HM, 0, 4 * ne * sizeof(double)));
  CK(cudaMemcpy2D(c->d.HM, 4 * sizeof(double), HM, 3 * sizeof(double), 3 * sizeof(double), ne, cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.t, t, ne * sizeof(long long), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.dt, dt, ne * sizeof(long long), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.X, X, 6 * ne * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.count, count, ne * sizeof(long long), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.qhat, qhat, ne * c->tab.Nst * 4 * sizeof(double), cudaMemcpyDefault));
  int rc0 = reset_sweep_state(c);
  if (rc0) return rc0;
  if ((rc0 = count_unfinished(c, nullptr))) return rc0;

  launch_products(c->tab, c->d, c->nsm, c->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->have_state = true;
  c->failed = false;
  c->fresh = false;
  c->adj_ready = false;
  return AW_OK;
}

int aw_get_node_arrays(aw_ctx* c, double* X, int64_t* t) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  CK(cudaStreamSynchronize(c->stream));
  if (X) CK(cudaMemcpy(X, c->d.nX, 2 * c->nn * sizeof(double), cudaMemcpyDefault));
  if (t) CK(cudaMemcpy(t, c->d.nt, c->nn * sizeof(long long), cudaMemcpyDefault));
  return AW_OK;
}

int aw_set_node_arrays(aw_ctx* c, const double* X, const int64_t* t) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !X || !t) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(c->d.nX, X, 2 * c->nn * sizeof(double), cudaMemcpyDefault));
  CK(cudaMemcpy(c->d.nt, t, c->nn * sizeof(long long), cudaMemcpyDefault));
  return AW_OK;
}

int aw_diagnostics(aw_ctx* c, double* out) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !out) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  int rc = sync_counters(c);
  if (rc) return rc;
  double g;
  std::memcpy(&g, &c->hcnt->gcl_bits, sizeof g);
  out[0] = g;
  out[1] = (double)c->hcnt->updates;
  out[2] = (double)c->hcnt->sweeps;
  out[3] = (double)c->hcnt->surfaces;
  return AW_OK;
}

int aw_sizes(aw_ctx* c, int64_t* out) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !out) return AW_ERR_INVALID_ARG;
  out[0] = c->ne; out[1] = c->nn; out[2] = c->ned; out[3] = c->tab.Nst; out[4] = c->sw_total;
  out[5] = c->u_total;
  return AW_OK;
}

int aw_profile_enable(aw_ctx* c, int on) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  int rc = sync_counters(c);
  if (rc) return rc;
  c->prof = on != 0;
  for (double& v : c->prof_ms) v = 0.0;
  c->prof_sweeps = 0;
  return AW_OK;
}

int aw_profile_read(aw_ctx* c, double* ms, int64_t* sweeps) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  int rc = sync_counters(c);
  if (rc) return rc;
  if (ms)
    for (int k = 0; k < kNumKernels; ++k) ms[k] = c->prof_ms[k];
  if (sweeps) *sweeps = c->prof_sweeps;
  return kNumKernels;
}

const char* aw_kernel_name(int k) { return kernel_name(k); }

int aw_measure_fp64_peak(double* gflops) {
  if (!gflops) return AW_ERR_INVALID_ARG;
  double v = measure_fp64_peak();
  if (!(v > 0)) return AW_ERR_CUDA;
  *gflops = v;
  return AW_OK;
}

int aw_schedule(aw_ctx* c, int mode, int64_t k) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || mode < 0 || mode > 2) return AW_ERR_INVALID_ARG;
  if (!c->have_mesh) return set_err(c, AW_ERR_STATE, "no mesh loaded");
  if (mode != 0 && c->cfg.gts) return set_err(c, AW_ERR_INVALID_ARG, "the schedule log is for local time stepping");
  CK(cudaStreamSynchronize(c->stream));
  if (mode == 1) {
    if (k < 1 || k > (1LL << 20)) return set_err(c, AW_ERR_INVALID_ARG, "schedule length must be in [1, 2^20]");
    long long* p = nullptr;
    int rc = dalloc(c, &p, (size_t)c->ne * k);
    if (rc) return rc;
    CK(cudaMemset(p, 0, (size_t)c->ne * k * sizeof(long long)));
    c->d_sched = p;
    c->d.sched_log = c->d_sched;
    c->d.sched_k = k;
  } else if (mode == 2 && !c->d_sched) {
    return set_err(c, AW_ERR_STATE, "no recorded schedule to replay");
  }
  c->d.sched_mode = mode;
  drop_graphs(c);  // the captured sweeps hold the old mode
  return AW_OK;
}

int aw_get_schedule(aw_ctx* c, int64_t* out) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !out) return AW_ERR_INVALID_ARG;
  if (!c->d_sched) return set_err(c, AW_ERR_STATE, "no recorded schedule");
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(out, c->d_sched, (size_t)c->ne * c->d.sched_k * sizeof(long long), cudaMemcpyDefault));
  return AW_OK;
}

int aw_adjoint_forward(aw_ctx* c, int64_t n_sweeps, int64_t ckpt_every) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || n_sweeps < 0 || ckpt_every < 1) return AW_ERR_INVALID_ARG;
  if (!c->have_state || c->failed) return set_err(c, AW_ERR_STATE, "no valid state (load a state first)");
  if (!c->fresh) return set_err(c, AW_ERR_STATE, "aw_adjoint_forward starts from a state just loaded");
  if (c->cfg.gts) return set_err(c, AW_ERR_INVALID_ARG, "the adjoint is for local time stepping");
  if (c->cfg.flux != 0) return set_err(c, AW_ERR_INVALID_ARG, "the adjoint covers the Rusanov-type flux");
  if (c->tab.Tsw > 0 || c->moving_wall)
    return set_err(c, AW_ERR_INVALID_ARG, "the adjoint covers neither moving walls, Kidder boundaries nor the global-step start-up");
  CK(cudaStreamSynchronize(c->stream));
  for (void* p : c->adj_allocs) cudaFree(p);
  c->adj_allocs.clear();
  c->ckpt.clear();
  c->slots.clear();
  c->adjv = Adj{};
  c->d_gxy = nullptr;
  c->adj_ready = false;
  int rc;
  const int64_t nck = n_sweeps / ckpt_every + 1;
  c->ckpt.resize(nck);
  for (auto& s : c->ckpt)
    if ((rc = snap_alloc(c, &s))) return rc;
  if ((rc = snap_alloc(c, &c->fin))) return rc;
  c->slots.resize(ckpt_every + 1);
  for (auto& s : c->slots)
    if ((rc = snap_alloc(c, &s))) return rc;
  c->last_seg_kept = false;
  if ((rc = snap_copy(c, c->ckpt[0], true))) return rc;
  // the last segment is the first one the reverse pass needs: keep its
  // sweep-start states now instead of recomputing them
  const int64_t last_s0 = n_sweeps > 0 ? (n_sweeps - 1) / ckpt_every * ckpt_every : 0;
  for (int64_t m = 1; m <= n_sweeps; ++m) {
    if ((rc = do_sweeps(c, 1, nullptr, false))) return rc;
    if (m % ckpt_every == 0 && (rc = snap_copy(c, c->ckpt[m / ckpt_every], true))) return rc;
    if (m > last_s0 && (rc = snap_copy(c, c->slots[m - last_s0], true))) return rc;
  }
  c->last_seg_kept = n_sweeps > 0;
  if ((rc = snap_copy(c, c->fin, true))) return rc;
  if ((rc = sync_counters(c))) return rc;
  if ((rc = check_device_error(c))) return rc;
  c->adj_n = n_sweeps;
  c->adj_k = ckpt_every;
  c->adj_ready = true;
  c->fresh = false;
  return AW_OK;
}

int aw_adjoint(aw_ctx* c, const double* dJdQ, const double* dJdX, const double* dJdxy, double* gQ0, double* gxy0) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c) return AW_ERR_INVALID_ARG;
  if (!c->adj_ready || c->failed) return set_err(c, AW_ERR_STATE, "no recorded forward run (call aw_adjoint_forward)");
  const size_t ne = c->ne, nn = c->nn, Nt = c->tab.Nt;
  int rc;
  Adj& a = c->adjv;
  if (!c->d_gxy) {
    void* p = nullptr;
    size_t nd[9] = {4 * ne, 4 * ne, 6 * ne, ne * 3 * Nt * Nt * 4, ne * Nt * 4, ne * 6 * Nt, 2 * nn, 2 * nn, 4 * ne};
    double** dst[9] = {&a.Qb, &a.QMb, &a.Xb, &a.trb, &a.avb, &a.vdb, &a.nXb, &a.nXnb, &a.gb};
    for (int k = 0; k < 9; ++k) {
      if ((rc = adj_alloc(c, &p, nd[k] * sizeof(double)))) return rc;
      *dst[k] = (double*)p;
    }
    if ((rc = adj_alloc(c, &p, 2 * nn * sizeof(double)))) return rc;
    c->d_gxy = (double*)p;
  }

  CK(cudaStreamSynchronize(c->stream));
  // seed with dJ / d(final state)
  if (dJdQ) CK(cudaMemcpyAsync(a.Qb, dJdQ, 4 * ne * sizeof(double), cudaMemcpyDefault, c->stream));
  else CK(cudaMemsetAsync(a.Qb, 0, 4 * ne * sizeof(double), c->stream));
  if (dJdX) CK(cudaMemcpyAsync(a.Xb, dJdX, 6 * ne * sizeof(double), cudaMemcpyDefault, c->stream));
  else CK(cudaMemsetAsync(a.Xb, 0, 6 * ne * sizeof(double), c->stream));
  if (dJdxy) CK(cudaMemcpyAsync(a.nXb, dJdxy, 2 * nn * sizeof(double), cudaMemcpyDefault, c->stream));
  else CK(cudaMemsetAsync(a.nXb, 0, 2 * nn * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.QMb, 0, 4 * ne * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.trb, 0, ne * 3 * Nt * Nt * 4 * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.avb, 0, ne * Nt * 4 * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.vdb, 0, ne * 6 * Nt * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.nXnb, 0, 2 * nn * sizeof(double), c->stream));
  CK(cudaMemsetAsync(a.gb, 0, 4 * ne * sizeof(double), c->stream));
  const int64_t n = c->adj_n, k = c->adj_k;
  const int64_t nseg = (n + k - 1) / k;
  for (int64_t seg = nseg - 1; seg >= 0; --seg) {
    const int64_t s0 = seg * k, s1 = std::min(s0 + k, n), len = s1 - s0;
    // recompute the segment from its checkpoint, keeping every sweep-start
    // state (the last segment's are kept by the forward run)
    if (!(seg == nseg - 1 && c->last_seg_kept)) {
      if ((rc = snap_copy(c, c->ckpt[seg], false))) return rc;
      for (int64_t j = 1; j <= len; ++j) {
        if ((rc = do_sweeps(c, 1, nullptr, false))) return rc;
        if ((rc = snap_copy(c, c->slots[j], true))) return rc;
      }
    }
    c->last_seg_kept = false;
    for (int64_t j = len - 1; j >= 0; --j) {
      // the sweep's lists and its reverse read the sweep-start state where
      // the snapshot holds it (they write only scratch lists and adjoints);
      // only the counters go back to the live block
      const aw_ctx::Snap& pre = j == 0 ? c->ckpt[seg] : c->slots[j];
      launch_adj_reset(c->d, pre.cnt, c->stream);
      const Dev pv = snap_view(c, pre);
      launch_phase_a_lists(c->tab, pv, c->nsm, c->stream);
      const Dev post = snap_view(c, c->slots[j + 1]);
      launch_adj_elem(c->tab, post, pv, a, c->nsm, c->stream, 0);
      launch_adj_phase_a(c->tab, pv, post, a, c->nsm, c->stream);
      CK(cudaGetLastError());
    }
  }
  // the pre-processing phase: reconstruction and predictor of every element
  launch_adj_elem(c->tab, snap_view(c, c->ckpt[0]), c->d, a, c->nsm, c->stream, 1);
  CK(cudaMemcpyAsync(c->d_gxy, a.nXb, 2 * nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  launch_adj_grad(c->d, a, c->d_gxy, c->nsm, c->stream);
  CK(cudaGetLastError());
  if ((rc = snap_copy(c, c->fin, false))) return rc;
  if ((rc = sync_counters(c))) return rc;
  if ((rc = check_device_error(c))) return rc;
  if (gQ0) CK(cudaMemcpy(gQ0, a.Qb, 4 * ne * sizeof(double), cudaMemcpyDefault));
  if (gxy0) CK(cudaMemcpy(gxy0, c->d_gxy, 2 * nn * sizeof(double), cudaMemcpyDefault));
  return AW_OK;
}

int aw_set_tiles(aw_ctx* c, const int32_t* tiles) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !tiles) return AW_ERR_INVALID_ARG;
  if (tiles[0] < 0 || tiles[0] > 1 || tiles[1] < 0 || tiles[1] > 1 || tiles[2] < 1 || tiles[2] > 64)
    return set_err(c, AW_ERR_INVALID_ARG, "tiles: recon_half and pred_wide are 0 or 1, blocks per SM in [1, 64]");
  CK(cudaStreamSynchronize(c->stream));
  c->tiles.recon_half = tiles[0];
  c->tiles.pred_wide = tiles[1];
  c->tiles.bpsm = tiles[2];
  drop_graphs(c);
  return AW_OK;
}

int aw_get_tiles(aw_ctx* c, int32_t* tiles) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || !tiles) return AW_ERR_INVALID_ARG;
  tiles[0] = c->tiles.recon_half;
  tiles[1] = c->tiles.pred_wide;
  tiles[2] = c->tiles.bpsm;
  return AW_OK;
}

int aw_autotune(aw_ctx* c, int64_t n_sweeps, double* ms, int32_t* best) {
  DeviceGuard dg_(c ? c->device : -1);
  if (!c || n_sweeps < 1) return AW_ERR_INVALID_ARG;
  if (!c->have_state || c->failed) return set_err(c, AW_ERR_STATE, "no valid state (load a state first)");
  CK(cudaStreamSynchronize(c->stream));
  std::vector<void*> owned;
  aw_ctx::Snap keep{};
  int rc = snap_alloc(c, &keep, &owned);
  auto done = [&](int code) {
    cudaStreamSynchronize(c->stream);
    for (void* p : owned) cudaFree(p);
    return code;
  };
  if (rc) return done(rc);
  const bool fresh = c->fresh;
  const bool prof = c->prof;
  c->prof = false;
  if ((rc = snap_copy(c, keep, true))) return done(rc);
  const Tiles start = c->tiles;
  Tiles best_t = start;
  double best_ms = 1e300;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  static const int kBpsm[3] = {4, 8, 16};
  for (int k = 0; k < 12; ++k) {  // candidate k: recon_half = k / 6, pred_wide = (k / 3) % 2, bpsm = kBpsm[k % 3]
    c->tiles.recon_half = k / 6;
    c->tiles.pred_wide = (k / 3) % 2;
    c->tiles.bpsm = kBpsm[k % 3];
    drop_graphs(c);
    // the first sweep captures this shape's graph; every candidate then times
    // the same sweeps from the same state
    if ((rc = snap_copy(c, keep, false)) || (rc = do_sweeps(c, 1, nullptr, false))) break;
    float t = 1e30f;
    for (int rep = 0; rep < 2 && !rc; ++rep) {  // the faster of two timed passes
      if ((rc = snap_copy(c, keep, false))) break;
      if (cudaEventRecord(e0, c->stream) != cudaSuccess) { rc = AW_ERR_CUDA; break; }
      if ((rc = do_sweeps(c, n_sweeps, nullptr, false))) break;
      float tr = 0.0f;
      if (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&tr, e0, e1) != cudaSuccess) {
        rc = set_err(c, AW_ERR_CUDA, "autotune: event timing failed");
        break;
      }
      t = std::min(t, tr);
    }
    if (rc) break;
    if (ms) ms[k] = t;
    if (t < best_ms) {
      best_ms = t;
      best_t = c->tiles;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tiles = rc ? start : best_t;
  drop_graphs(c);
  int rc2 = snap_copy(c, keep, false);
  c->prof = prof;
  c->fresh = fresh;
  if (rc || rc2) return done(rc ? rc : rc2);
  if ((rc = sync_counters(c))) return done(rc);
  if ((rc = check_device_error(c))) return done(rc);
  if (best) {
    best[0] = c->tiles.recon_half;
    best[1] = c->tiles.pred_wide;
    best[2] = c->tiles.bpsm;
  }
  return done(AW_OK);
}

int aw_adjoint_selftest(int order_M, uint64_t seed, double* report) {
  if (order_M < 1 || order_M > kMaxM || !report) return AW_ERR_INVALID_ARG;
  aw_ctx tmp;
  tmp.cfg.order_M = order_M;
  tmp.cfg.gamma = 1.4;
  tmp.cfg.cfl = 0.5;
  tmp.cfg.time_quantum_log2 = 20;
  tmp.cfg.t_end = 1.0;
  int rc = build_tab(&tmp);
  if (rc) return rc;
  return adjoint_selftest(tmp.tab, (unsigned long long)seed, report);
}

}  // extern "C"

