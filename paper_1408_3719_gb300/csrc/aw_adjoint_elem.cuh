// Element-local pieces of one LTS sweep, each with its hand-written reverse
// (the discrete adjoint of the same arithmetic):
//   recon_fwd / recon_rev   virtual data -> WENO nodal values w_h (eqs.
//                           intConsRec, weno; characteristic weights R10)
//   pred_fwd / pred_rev     w_h, vertices, dt -> space-time predictor and its
//                           derived tables (eqs. PDECG, pdef, CGfinal, Jac,
//                           newVertPos)
//   edge_fwd / edge_rev     one swept edge surface: Gauss quadrature of the
//                           Rusanov ALE flux (eqs. spacetimenodes, rusanov, STint)
//   node_fwd / node_rev     node solver NS_cs (eqs. eqnNScs, NodesVel, newVertex)
// The integer schedule (ready sets, time steps in ticks) and the mesh
// pre-processing (stencils, wall normals) are held fixed: the reverse
// functions differentiate the sweep map for that schedule.
//
// The reconstruction and predictor pieces run on a team: the 32 lanes of a
// warp on the GPU (work arrays in shared memory, loops strided over the
// lanes, scatters by shared-memory atomics), or one serial rank on the host,
// where the library checks every reverse against central differences of its
// forward.  All functions are __host__ __device__.
#pragma once
#include <cmath>

#include "aw_internal.h"

#ifdef __CUDACC__
#define AW_HD __host__ __device__
#else
#define AW_HD
#endif

namespace aw {
namespace adj {

template <int M>
struct Sz {
  static constexpr int Mc = (M + 1) * (M + 2) / 2, Nt = M + 1, Nst = Mc * Nt, NU = Mc - 1, NE = 2 * Mc;
  static constexpr int MaxU = kNSten * (NE - 1);
  static constexpr int NL = NU * (NU + 1) / 2;
  static constexpr int NN = NL + 4 * NU;  // normal matrix (lower triangle) and right-hand sides
};

// one serial rank
struct TeamSerial {
  int rank = 0, size = 1;
  AW_HD void sync() const {}
  AW_HD double sum(double v) const { return v; }
  AW_HD void add(double* p, double v) const { *p += v; }
  AW_HD int any(int f) const { return f; }
};

// the 32 lanes of a warp; every lane calls sync, sum and any
struct TeamWarp {
  int rank, size;
  AW_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncwarp();
#endif
  }
  AW_HD double sum(double v) const {
#ifdef __CUDA_ARCH__
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
#endif
    return v;
  }
  AW_HD void add(double* p, double v) const {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
  }
  AW_HD int any(int f) const {
#ifdef __CUDA_ARCH__
    return __any_sync(0xffffffffu, f);
#else
    return f;
#endif
  }
};

// the threads of a block; red = shared scratch of one double per warp; every
// thread calls sync, sum and any
struct TeamBlock {
  int rank, size;
  double* red;
  AW_HD void sync() const {
#ifdef __CUDA_ARCH__
    __syncthreads();
#endif
  }
  AW_HD double sum(double v) const {
#ifdef __CUDA_ARCH__
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((rank & 31) == 0) red[rank >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (size >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
#else
    return v;
#endif
  }
  AW_HD void add(double* p, double v) const {
#ifdef __CUDA_ARCH__
    atomicAdd(p, v);
#else
    *p += v;
#endif
  }
  AW_HD int any(int f) const {
#ifdef __CUDA_ARCH__
    return __syncthreads_or(f);
#else
    return f;
#endif
  }
};

AW_HD inline double tri_area(const double* X) {
  return 0.5 * ((X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0]));
}
// adds s * d|T|/dX to Xb
AW_HD inline void tri_area_rev(const double* X, double s, double* Xb) {
  Xb[0] += 0.5 * s * (X[3] - X[5]);
  Xb[1] += 0.5 * s * (X[4] - X[2]);
  Xb[2] += 0.5 * s * (X[5] - X[1]);
  Xb[3] += 0.5 * s * (X[0] - X[4]);
  Xb[4] += 0.5 * s * (X[1] - X[3]);
  Xb[5] += 0.5 * s * (X[2] - X[0]);
}

// Averages of the graded monomials (mono's order) over the straight triangle
// with vertices (x_k, y_k), in closed form: with the centroid c and the
// offsets u_k = v_k - c (sum u_k = 0), the second central moments are
// S = (1/12) sum u u^T and the third (1/30) sum u (x) u (x) u; e.g.
// E[x^2] = c_x^2 + S_xx, E[x^2 y] = c_y (c_x^2 + S_xx) + 2 c_x S_xy + T_xxy.
template <int M>
AW_HD inline void tri_monomial_avgs(const double* x, const double* y, double* row) {
  const double cx = (x[0] + x[1] + x[2]) * (1.0 / 3.0), cy = (y[0] + y[1] + y[2]) * (1.0 / 3.0);
  row[0] = cx;
  row[1] = cy;
  if (M >= 2) {
    double ux[3], uy[3];
    for (int k = 0; k < 3; ++k) {
      ux[k] = x[k] - cx;
      uy[k] = y[k] - cy;
    }
    const double sxx = (ux[0] * ux[0] + ux[1] * ux[1] + ux[2] * ux[2]) * (1.0 / 12.0);
    const double sxy = (ux[0] * uy[0] + ux[1] * uy[1] + ux[2] * uy[2]) * (1.0 / 12.0);
    const double syy = (uy[0] * uy[0] + uy[1] * uy[1] + uy[2] * uy[2]) * (1.0 / 12.0);
    row[2] = cx * cx + sxx;
    row[3] = cx * cy + sxy;
    row[4] = cy * cy + syy;
    if (M >= 3) {
      double txxx = 0.0, txxy = 0.0, txyy = 0.0, tyyy = 0.0;
      for (int k = 0; k < 3; ++k) {
        const double xx = ux[k] * ux[k], yy = uy[k] * uy[k];
        txxx += xx * ux[k];
        txxy += xx * uy[k];
        txyy += yy * ux[k];
        tyyy += yy * uy[k];
      }
      const double c30 = 1.0 / 30.0;
      row[5] = cx * (cx * cx + 3.0 * sxx) + txxx * c30;
      row[6] = cy * (cx * cx + sxx) + 2.0 * cx * sxy + txxy * c30;
      row[7] = cx * (cy * cy + syy) + 2.0 * cy * sxy + txyy * c30;
      row[8] = cy * (cy * cy + 3.0 * syy) + tyyy * c30;
    }
  }
}

// Reverse of tri_monomial_avgs: adds sum_a rb[a] d row_a / d x_k to xb[k]
// (and likewise yb); d c_x / d x_k = 1/3, d S_xx / d x_k = u_k / 6,
// d (sum u_x^3) / d x_k = 3 u_k^2 - 12 S_xx, and so on (sum u = 0).
template <int M>
AW_HD inline void tri_monomial_avgs_rev(const double* x, const double* y, const double* rb, double* xb, double* yb) {
  const double cx = (x[0] + x[1] + x[2]) * (1.0 / 3.0), cy = (y[0] + y[1] + y[2]) * (1.0 / 3.0);
  double ux[3], uy[3];
  for (int k = 0; k < 3; ++k) {
    ux[k] = x[k] - cx;
    uy[k] = y[k] - cy;
  }
  const double sxx = (ux[0] * ux[0] + ux[1] * ux[1] + ux[2] * ux[2]) * (1.0 / 12.0);
  const double sxy = (ux[0] * uy[0] + ux[1] * uy[1] + ux[2] * uy[2]) * (1.0 / 12.0);
  const double syy = (uy[0] * uy[0] + uy[1] * uy[1] + uy[2] * uy[2]) * (1.0 / 12.0);
  const double t3 = 1.0 / 3.0, c30 = 1.0 / 30.0;
  for (int k = 0; k < 3; ++k) {
    double gx = rb[0] * t3, gy = rb[1] * t3;
    if (M >= 2) {
      gx += rb[2] * (2.0 * cx * t3 + ux[k] * (1.0 / 6.0)) + rb[3] * (cy * t3 + uy[k] * (1.0 / 12.0));
      gy += rb[3] * (cx * t3 + ux[k] * (1.0 / 12.0)) + rb[4] * (2.0 * cy * t3 + uy[k] * (1.0 / 6.0));
    }
    if (M >= 3) {
      const double xy = ux[k] * uy[k];
      gx += rb[5] * (cx * cx + sxx + 0.5 * cx * ux[k] + (3.0 * ux[k] * ux[k] - 12.0 * sxx) * c30);
      gx += rb[6] * (2.0 * cx * cy * t3 + (cy * ux[k] + cx * uy[k]) * (1.0 / 6.0) + 2.0 * sxy * t3 +
                     (2.0 * xy - 8.0 * sxy) * c30);
      gx += rb[7] * ((cy * cy + syy) * t3 + cy * uy[k] * (1.0 / 6.0) + (uy[k] * uy[k] - 4.0 * syy) * c30);
      gy += rb[6] * ((cx * cx + sxx) * t3 + cx * ux[k] * (1.0 / 6.0) + (ux[k] * ux[k] - 4.0 * sxx) * c30);
      gy += rb[7] * (2.0 * cx * cy * t3 + (cx * uy[k] + cy * ux[k]) * (1.0 / 6.0) + 2.0 * sxy * t3 +
                     (2.0 * xy - 8.0 * sxy) * c30);
      gy += rb[8] * (cy * cy + syy + 0.5 * cy * uy[k] + (3.0 * uy[k] * uy[k] - 12.0 * syy) * c30);
    }
    xb[k] += gx;
    yb[k] += gy;
  }
}

// Euler fluxes f, g of one state and the reverse (adds to qb)
AW_HD inline void euler_fg(double gm1, const double* q, double* f, double* g) {
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  f[0] = q[1]; f[1] = q[1] * u + p; f[2] = q[1] * v; f[3] = u * (q[3] + p);
  g[0] = q[2]; g[1] = q[2] * u; g[2] = q[2] * v + p; g[3] = v * (q[3] + p);
}
AW_HD inline void euler_fg_rev(double gm1, const double* q, const double* fb, const double* gb, double* qb) {
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  double ub = fb[1] * q[1] + fb[3] * (q[3] + p) + gb[1] * q[2];
  double vb = fb[2] * q[1] + gb[2] * q[2] + gb[3] * (q[3] + p);
  const double pb = fb[1] + fb[3] * u + gb[2] + gb[3] * v;
  double q1b = fb[0] + fb[1] * u + fb[2] * v;
  double q2b = gb[0] + gb[1] * u + gb[2] * v;
  double q3b = fb[3] * u + gb[3] * v;
  q3b += gm1 * pb;
  q1b -= 0.5 * gm1 * pb * u;
  q2b -= 0.5 * gm1 * pb * v;
  ub -= 0.5 * gm1 * pb * q[1];
  vb -= 0.5 * gm1 * pb * q[2];
  q1b += ub * ir;
  q2b += vb * ir;
  const double irb = ub * q[1] + vb * q[2];
  qb[0] -= irb * ir * ir;
  qb[1] += q1b;
  qb[2] += q2b;
  qb[3] += q3b;
}

AW_HD inline double pressure_of(double gm1, const double* q) {
  return gm1 * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

// ---------------------------------------------------------------------------
// Reconstruction of one element
// ---------------------------------------------------------------------------
template <int M>
struct ReconIn {
  using S = Sz<M>;
  double X[6], Q[4];                 // own vertices and average (after the update)
  double Xv[S::MaxU][6];             // members' virtual vertices, periodic shift applied
  double Qv[S::MaxU][4];             // members' virtual averages
  int nU;                            // distinct stencil members
  unsigned char st[kNSten][S::NE];   // stencil rows: 0 = the element, u + 1 = member u
  signed char ok[kNSten];
};

template <int M>
struct ReconTape {
  using S = Sz<M>;
  double ja, jb, jc, jd, idet, J[4];
  double rows[S::MaxU + 1][S::NU + 4];
  double Nrm[kNSten][S::NN];     // normal equations: lower triangle, then right-hand sides
  double Lf[kNSten][S::NL];      // Cholesky factors, diagonal stored as 1 / L_aa
  double c[kNSten][S::NU][4];
  double gx, gy, gn, nx, ny;
  double R[16], Lm[16];
  double ch[kNSten][S::NU][4];
  double y[kNSten][4][S::NU];    // SigU ch
  double e1[kNSten][4], om[kNSten][4], tot[4];
  double wc[S::NU][4], cv[S::NU][4];
  double w[S::Mc][4];            // nodal w_h
  int limited;                   // the positivity scaling would change w_h
};

// reverse scratch of the reconstruction
template <int M>
struct ReconRev {
  using S = Sz<M>;
  double cvb[S::NU][4], wcb[S::NU][4], Rb[16], Lb[16];
  double omtb[kNSten][4], dot[4];
  double chb[kNSten][S::NU][4], cb[kNSten][S::NU][4];
  double lam[kNSten][S::NU][4];
  double nsym[kNSten][S::NU][S::NU];  // -(lam c^T + c lam^T): adjoint of the symmetric normal matrix
  double rowb[S::MaxU + 1][S::NU + 4];  // adjoint of every member row
};

template <int M>
AW_HD inline void chol_solve(const double* Lf, double* y) {
  constexpr int NU = Sz<M>::NU;
  for (int a = 0; a < NU; ++a) {
    double acc = y[a];
    for (int k = 0; k < a; ++k) acc -= Lf[a * (a + 1) / 2 + k] * y[k];
    y[a] = acc * Lf[a * (a + 1) / 2 + a];
  }
  for (int a = NU - 1; a >= 0; --a) {
    double acc = y[a];
    for (int k = a + 1; k < NU; ++k) acc -= Lf[k * (k + 1) / 2 + a] * y[k];
    y[a] = acc * Lf[a * (a + 1) / 2 + a];
  }
}

template <int M, class Tm>
AW_HD void recon_fwd(const Tab& T, const ReconIn<M>& in, ReconTape<M>& tp, const Tm& tm) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, NU = S::NU, NE = S::NE, NL = S::NL, NN = S::NN;
  const double* X = in.X;
  const double ja = X[2] - X[0], jb = X[4] - X[0], jc = X[3] - X[1], jd = X[5] - X[1];
  const double idet = 1.0 / (ja * jd - jb * jc);
  const double J[4] = {jd * idet, -jb * idet, -jc * idet, ja * idet};
  if (tm.rank == 0) {
    tp.ja = ja; tp.jb = jb; tp.jc = jc; tp.jd = jd; tp.idet = idet;
    for (int k = 0; k < 4; ++k) tp.J[k] = J[k];
  }
  for (int u = tm.rank; u < in.nU; u += tm.size) {
    double xr[3], yr[3];
    for (int k = 0; k < 3; ++k) {
      const double px = in.Xv[u][2 * k] - X[0], py = in.Xv[u][2 * k + 1] - X[1];
      xr[k] = J[0] * px + J[1] * py - (1.0 / 3.0);
      yr[k] = J[2] * px + J[3] * py - (1.0 / 3.0);
    }
    double row[NU];
    tri_monomial_avgs<M>(xr, yr, row);
    double* dst = tp.rows[u + 1];
    for (int a = 0; a < NU; ++a) dst[a] = row[a] - T.mbar[a];
    for (int v = 0; v < 4; ++v) dst[NU + v] = in.Qv[u][v] - in.Q[v];
  }
  tm.sync();
  // normal equations of every stencil
  for (int it = tm.rank; it < kNSten * NN; it += tm.size) {
    const int s = it / NN, q = it % NN;
    if (!in.ok[s]) continue;
    int a, b;
    if (q < NL) {
      a = 0;
      while ((a + 1) * (a + 2) / 2 <= q) ++a;
      b = q - a * (a + 1) / 2;
    } else {
      a = (q - NL) / 4;
      b = NU + (q - NL) % 4;
    }
    double acc = 0.0;
    for (int m = 1; m < NE; ++m) {
      const double* r = tp.rows[in.st[s][m]];
      acc += r[a] * r[b];
    }
    tp.Nrm[s][q] = acc;
  }
  tm.sync();
  for (int s = tm.rank; s < kNSten; s += tm.size) {
    if (!in.ok[s]) continue;
    double Lw[NU][NU];
    for (int a = 0; a < NU; ++a)
      for (int bb = 0; bb <= a; ++bb) Lw[a][bb] = tp.Nrm[s][a * (a + 1) / 2 + bb];
    for (int a = 0; a < NU; ++a) {
      double dd = Lw[a][a];
      for (int k = 0; k < a; ++k) dd -= Lw[a][k] * Lw[a][k];
      const double il = 1.0 / sqrt(dd);
      Lw[a][a] = il;
      for (int bb = a + 1; bb < NU; ++bb) {
        double v = Lw[bb][a];
        for (int k = 0; k < a; ++k) v -= Lw[bb][k] * Lw[a][k];
        Lw[bb][a] = v * il;
      }
    }
    for (int a = 0; a < NU; ++a)
      for (int bb = 0; bb <= a; ++bb) tp.Lf[s][a * (a + 1) / 2 + bb] = Lw[a][bb];
  }
  tm.sync();
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, v = it % 4;
    if (!in.ok[s]) continue;
    double y[NU];
    for (int a = 0; a < NU; ++a) y[a] = tp.Nrm[s][NL + a * 4 + v];
    chol_solve<M>(tp.Lf[s], y);
    for (int a = 0; a < NU; ++a) tp.c[s][a][v] = y[a];
  }
  tm.sync();
  // characteristic fields along the density gradient of the central stencil
  if (tm.rank == 0) {
    tp.gx = tp.c[0][0][0] * J[0] + tp.c[0][1][0] * J[2];
    tp.gy = tp.c[0][0][0] * J[1] + tp.c[0][1][0] * J[3];
    tp.gn = sqrt(tp.gx * tp.gx + tp.gy * tp.gy);
    tp.nx = 1.0; tp.ny = 0.0;
    if (tp.gn > 0.0) {  // reciprocals, not divides: this runs on one rank
      const double ign = 1.0 / tp.gn;
      tp.nx = tp.gx * ign;
      tp.ny = tp.gy * ign;
    }
    const double g = T.gamma, rho = in.Q[0], ir = 1.0 / rho, u = in.Q[1] * ir, v = in.Q[2] * ir;
    const double nx = tp.nx, ny = tp.ny;
    const double p = (g - 1.0) * (in.Q[3] - 0.5 * rho * (u * u + v * v));
    const double a = sqrt(g * p * ir), H = (in.Q[3] + p) * ir, un = u * nx + v * ny, ut = -u * ny + v * nx;
    const double ia = 1.0 / a, q2 = 0.5 * (u * u + v * v), b1 = (g - 1.0) * ia * ia, b2 = b1 * q2;
    double* R = tp.R;
    double* Lm = tp.Lm;
    R[0] = 1; R[1] = 1; R[2] = 0; R[3] = 1;
    R[4] = u - a * nx; R[5] = u; R[6] = -ny; R[7] = u + a * nx;
    R[8] = v - a * ny; R[9] = v; R[10] = nx; R[11] = v + a * ny;
    R[12] = H - a * un; R[13] = q2; R[14] = ut; R[15] = H + a * un;
    Lm[0] = 0.5 * (b2 + un * ia); Lm[1] = -0.5 * (b1 * u + nx * ia); Lm[2] = -0.5 * (b1 * v + ny * ia); Lm[3] = 0.5 * b1;
    Lm[4] = 1.0 - b2; Lm[5] = b1 * u; Lm[6] = b1 * v; Lm[7] = -b1;
    Lm[8] = -ut; Lm[9] = -ny; Lm[10] = nx; Lm[11] = 0.0;
    Lm[12] = 0.5 * (b2 - un * ia); Lm[13] = -0.5 * (b1 * u - nx * ia); Lm[14] = -0.5 * (b1 * v - ny * ia); Lm[15] = 0.5 * b1;
  }
  tm.sync();
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, r = it % 4;
    if (!in.ok[s]) continue;
    const double* Lr = tp.Lm + 4 * r;
    for (int l = 0; l < NU; ++l)
      tp.ch[s][l][r] = Lr[0] * tp.c[s][l][0] + Lr[1] * tp.c[s][l][1] + Lr[2] * tp.c[s][l][2] + Lr[3] * tp.c[s][l][3];
    double sg = 0.0;
    for (int a = 0; a < NU; ++a) {
      double acc = 0.0;
      for (int bb = a; bb < NU; ++bb) acc += T.SigU[a][bb] * tp.ch[s][bb][r];
      tp.y[s][r][a] = acc;
      sg += acc * acc;
    }
    tp.e1[s][r] = sg + 1e-14;
  }
  tm.sync();
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, r = it % 4;
    tp.om[s][r] = 0.0;
    if (!in.ok[s]) continue;
    const double e1 = tp.e1[s][r], e2 = e1 * e1, e4 = e2 * e2, e8 = e4 * e4;
    tp.om[s][r] = (s == 0 ? 1e5 : 1.0) / e8;
  }
  tm.sync();
  for (int r = tm.rank; r < 4; r += tm.size) {
    double tot = 0.0;
    for (int s = 0; s < kNSten; ++s)
      if (in.ok[s]) tot += tp.om[s][r];
    tp.tot[r] = tot;
  }
  tm.sync();
  for (int it = tm.rank; it < NU * 4; it += tm.size) {
    const int l = it / 4, r = it % 4;
    const double itot = 1.0 / tp.tot[r];
    double acc = 0.0;
    for (int s = 0; s < kNSten; ++s)
      if (in.ok[s]) acc += (tp.om[s][r] * itot) * tp.ch[s][l][r];
    tp.wc[l][r] = acc;
  }
  tm.sync();
  for (int it = tm.rank; it < NU * 4; it += tm.size) {
    const int l = it / 4, v = it % 4;
    const double* Rv = tp.R + 4 * v;
    tp.cv[l][v] = Rv[0] * tp.wc[l][0] + Rv[1] * tp.wc[l][1] + Rv[2] * tp.wc[l][2] + Rv[3] * tp.wc[l][3];
  }
  tm.sync();
  for (int it = tm.rank; it < Mc * 4; it += tm.size) {
    const int s = it / 4, v = it % 4;
    double acc = in.Q[v];
    for (int l = 0; l < NU; ++l) acc += T.Bnod[s][l] * tp.cv[l][v];
    tp.w[s][v] = acc;
  }
  tm.sync();
  // the positivity scaling (R11) is a kink: the reverse reports where it acts
  const double gm1 = T.gamma - 1.0, rho_min = 1e-8 * in.Q[0], p_min = 1e-8 * pressure_of(gm1, in.Q);
  int lim = 0;
  for (int s = tm.rank; s < Mc; s += tm.size)
    if (tp.w[s][0] < rho_min || pressure_of(gm1, tp.w[s]) < p_min) lim = 1;
  lim = tm.any(lim);
  if (tm.rank == 0) tp.limited = lim;
  tm.sync();
}

// Reverse of recon_fwd: wb = dJ/dw (Mc x 4); adds to Xb (6), Qb (4) of the
// element (rank 0 writes them) and to Xvb, Qvb of the members (zeroed by the
// caller; each member's row is written by one rank).
template <int M, class Tm>
AW_HD void recon_rev(const Tab& T, const ReconIn<M>& in, const ReconTape<M>& tp, const double (*wb)[4], double* Xb,
                     double* Qb, double (*Xvb)[6], double (*Qvb)[4], ReconRev<M>& sc, const Tm& tm) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, NU = S::NU, NE = S::NE;
  double pQ[4] = {0, 0, 0, 0}, pX[6] = {0, 0, 0, 0, 0, 0}, pJ[4] = {0, 0, 0, 0};  // this rank's partial sums
  // w = Q + Bnod cv
  for (int v = tm.rank; v < 4; v += tm.size) {
    double acc = 0.0;
    for (int s = 0; s < Mc; ++s) acc += wb[s][v];
    pQ[v] += acc;
  }
  for (int it = tm.rank; it < NU * 4; it += tm.size) {
    const int l = it / 4, v = it % 4;
    double acc = 0.0;
    for (int s = 0; s < Mc; ++s) acc += T.Bnod[s][l] * wb[s][v];
    sc.cvb[l][v] = acc;
  }
  tm.sync();
  // cv = R wc
  for (int it = tm.rank; it < NU * 4; it += tm.size) {
    const int l = it / 4, r = it % 4;
    double acc = 0.0;
    for (int v = 0; v < 4; ++v) acc += tp.R[4 * v + r] * sc.cvb[l][v];
    sc.wcb[l][r] = acc;
  }
  for (int it = tm.rank; it < 16; it += tm.size) {
    const int v = it / 4, r = it % 4;
    double acc = 0.0;
    for (int l = 0; l < NU; ++l) acc += sc.cvb[l][v] * tp.wc[l][r];
    sc.Rb[4 * v + r] = acc;
  }
  tm.sync();
  // nonlinear weights: wc = sum_s om_s / tot ch_s
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, r = it % 4;
    double acc = 0.0;
    if (in.ok[s])
      for (int l = 0; l < NU; ++l) acc += sc.wcb[l][r] * tp.ch[s][l][r];
    sc.omtb[s][r] = acc;
  }
  tm.sync();
  for (int r = tm.rank; r < 4; r += tm.size) {
    const double itot = 1.0 / tp.tot[r];
    double dot = 0.0;
    for (int s = 0; s < kNSten; ++s)
      if (in.ok[s]) dot += sc.omtb[s][r] * (tp.om[s][r] * itot);
    sc.dot[r] = dot;
  }
  tm.sync();
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, r = it % 4;
    if (!in.ok[s]) {
      for (int l = 0; l < NU; ++l) sc.chb[s][l][r] = 0.0;
      continue;
    }
    const double itot = 1.0 / tp.tot[r];
    const double omt = tp.om[s][r] * itot;
    for (int l = 0; l < NU; ++l) sc.chb[s][l][r] = omt * sc.wcb[l][r];
    const double omb = (sc.omtb[s][r] - sc.dot[r]) * itot;
    const double sigb = omb * (-8.0 * tp.om[s][r] / tp.e1[s][r]);
    // sigma = sum_a y_a^2, y = SigU ch
    for (int a = 0; a < NU; ++a) {
      const double yb = 2.0 * tp.y[s][r][a] * sigb;
      for (int bb = a; bb < NU; ++bb) sc.chb[s][bb][r] += T.SigU[a][bb] * yb;
    }
  }
  tm.sync();
  // ch = Lm c
  for (int it = tm.rank; it < kNSten * NU * 4; it += tm.size) {
    const int s = it / (NU * 4), l = (it / 4) % NU, v = it % 4;
    double acc = 0.0;
    if (in.ok[s])
      for (int r = 0; r < 4; ++r) acc += tp.Lm[4 * r + v] * sc.chb[s][l][r];
    sc.cb[s][l][v] = acc;
  }
  for (int it = tm.rank; it < 16; it += tm.size) {
    const int r = it / 4, v = it % 4;
    double acc = 0.0;
    for (int s = 0; s < kNSten; ++s)
      if (in.ok[s])
        for (int l = 0; l < NU; ++l) acc += sc.chb[s][l][r] * tp.c[s][l][v];
    sc.Lb[4 * r + v] = acc;
  }
  tm.sync();
  // eigenvectors of the direction n and the state Q, then n = g / |g|
  if (tm.rank == 0) {
    double nxb = 0.0, nyb = 0.0;
    const double g = T.gamma, rho = in.Q[0], irho = 1.0 / rho, u = in.Q[1] * irho, v = in.Q[2] * irho;
    const double nx = tp.nx, ny = tp.ny;
    const double p = (g - 1.0) * (in.Q[3] - 0.5 * rho * (u * u + v * v));
    const double a = sqrt(g * p * irho), ia = 1.0 / a, H = (in.Q[3] + p) * irho, un = u * nx + v * ny;
    const double q2 = 0.5 * (u * u + v * v), b1 = (g - 1.0) * ia * ia;
    double ub = 0, vb = 0, ab = 0, Hb = 0, unb = 0, utb = 0, q2b = 0, b1b = 0, b2b = 0, iab = 0;
    const double* R_ = sc.Rb;
    ub += R_[4]; ab -= R_[4] * nx; nxb -= R_[4] * a;
    ub += R_[5];
    nyb -= R_[6];
    ub += R_[7]; ab += R_[7] * nx; nxb += R_[7] * a;
    vb += R_[8]; ab -= R_[8] * ny; nyb -= R_[8] * a;
    vb += R_[9];
    nxb += R_[10];
    vb += R_[11]; ab += R_[11] * ny; nyb += R_[11] * a;
    Hb += R_[12]; ab -= R_[12] * un; unb -= R_[12] * a;
    q2b += R_[13];
    utb += R_[14];
    Hb += R_[15]; ab += R_[15] * un; unb += R_[15] * a;
    const double* L_ = sc.Lb;
    b2b += 0.5 * L_[0]; unb += 0.5 * L_[0] * ia; iab += 0.5 * L_[0] * un;
    b1b -= 0.5 * L_[1] * u; ub -= 0.5 * L_[1] * b1; nxb -= 0.5 * L_[1] * ia; iab -= 0.5 * L_[1] * nx;
    b1b -= 0.5 * L_[2] * v; vb -= 0.5 * L_[2] * b1; nyb -= 0.5 * L_[2] * ia; iab -= 0.5 * L_[2] * ny;
    b1b += 0.5 * L_[3];
    b2b -= L_[4];
    b1b += L_[5] * u; ub += L_[5] * b1;
    b1b += L_[6] * v; vb += L_[6] * b1;
    b1b -= L_[7];
    utb -= L_[8];
    nyb -= L_[9];
    nxb += L_[10];
    b2b += 0.5 * L_[12]; unb -= 0.5 * L_[12] * ia; iab -= 0.5 * L_[12] * un;
    b1b -= 0.5 * L_[13] * u; ub -= 0.5 * L_[13] * b1; nxb += 0.5 * L_[13] * ia; iab += 0.5 * L_[13] * nx;
    b1b -= 0.5 * L_[14] * v; vb -= 0.5 * L_[14] * b1; nyb += 0.5 * L_[14] * ia; iab += 0.5 * L_[14] * ny;
    b1b += 0.5 * L_[15];
    // b2 = b1 q2, b1 = (g-1)/a^2, ia = 1/a
    b1b += b2b * q2; q2b += b2b * b1;
    ab += b1b * (-2.0 * b1 * ia);
    ab -= iab * ia * ia;
    // q2, un, ut
    ub += q2b * u; vb += q2b * v;
    ub += unb * nx; vb += unb * ny; nxb += unb * u; nyb += unb * v;
    ub -= utb * ny; vb += utb * nx; nyb -= utb * u; nxb += utb * v;
    // H = (E + p)/rho, a = sqrt(g p / rho)
    double rhob = 0.0, pb = 0.0, Eb = 0.0;
    Eb += Hb * irho; pb += Hb * irho; rhob -= Hb * H * irho;
    pb += ab * g * 0.5 * ia * irho; rhob -= ab * a * 0.5 * irho;
    // p = (g-1)(E - rho (u^2+v^2)/2)
    Eb += pb * (g - 1.0); rhob -= pb * (g - 1.0) * 0.5 * (u * u + v * v);
    ub -= pb * (g - 1.0) * rho * u; vb -= pb * (g - 1.0) * rho * v;
    // u = Q1 / rho, v = Q2 / rho
    pQ[1] += ub * irho; rhob -= ub * u * irho;
    pQ[2] += vb * irho; rhob -= vb * v * irho;
    pQ[0] += rhob;
    pQ[3] += Eb;
    if (tp.gn > 0.0) {
      const double dn = tp.nx * nxb + tp.ny * nyb, ign = 1.0 / tp.gn;
      const double gxb = (nxb - tp.nx * dn) * ign, gyb = (nyb - tp.ny * dn) * ign;
      sc.cb[0][0][0] += gxb * tp.J[0] + gyb * tp.J[1];
      sc.cb[0][1][0] += gxb * tp.J[2] + gyb * tp.J[3];
      pJ[0] += gxb * tp.c[0][0][0];
      pJ[2] += gxb * tp.c[0][1][0];
      pJ[1] += gyb * tp.c[0][0][0];
      pJ[3] += gyb * tp.c[0][1][0];
    }
  }
  tm.sync();
  // least-squares solves: c = N^-1 b, N = sum r r^T, b = sum r rhs^T
  for (int it = tm.rank; it < kNSten * 4; it += tm.size) {
    const int s = it / 4, v = it % 4;
    if (!in.ok[s]) continue;
    double y[NU];
    for (int a = 0; a < NU; ++a) y[a] = sc.cb[s][a][v];
    chol_solve<M>(tp.Lf[s], y);
    for (int a = 0; a < NU; ++a) sc.lam[s][a][v] = y[a];
  }
  tm.sync();
  for (int it = tm.rank; it < kNSten * NU * NU; it += tm.size) {
    const int s = it / (NU * NU), k = (it / NU) % NU, bb = it % NU;
    if (!in.ok[s]) continue;
    double acc = 0.0;
    for (int v = 0; v < 4; ++v) acc -= sc.lam[s][k][v] * tp.c[s][bb][v] + sc.lam[s][bb][v] * tp.c[s][k][v];
    sc.nsym[s][k][bb] = acc;
  }
  tm.sync();
  // adjoint of every member row: the contributions of each stencil entry,
  // one item per (stencil, entry, row component), summed in shared memory
  for (int k = tm.rank; k < (in.nU + 1) * (NU + 4); k += tm.size) (&sc.rowb[0][0])[k] = 0.0;
  tm.sync();
  for (int it = tm.rank; it < kNSten * (NE - 1) * (NU + 4); it += tm.size) {
    const int s = it / ((NE - 1) * (NU + 4)), m = 1 + (it / (NU + 4)) % (NE - 1), k = it % (NU + 4);
    if (!in.ok[s]) continue;
    const int ri = in.st[s][m];
    const double* r = tp.rows[ri];
    double acc = 0.0;
    if (k < NU) {
      for (int bb = 0; bb < NU; ++bb) acc += sc.nsym[s][k][bb] * r[bb];
      for (int v = 0; v < 4; ++v) acc += sc.lam[s][k][v] * r[NU + v];
    } else {
      for (int a = 0; a < NU; ++a) acc += sc.lam[s][a][k - NU] * r[a];
    }
    tm.add(&sc.rowb[ri][k], acc);
  }
  tm.sync();
  // reverse of each row: basis averages over the virtual member, Qv - Q
  const double* X = in.X;
  const double* J = tp.J;
  for (int u = tm.rank; u < in.nU; u += tm.size) {
    const double* rb = sc.rowb[u + 1];
    for (int v = 0; v < 4; ++v) {
      Qvb[u][v] += rb[NU + v];
      pQ[v] -= rb[NU + v];
    }
    double px[3], py[3], xr[3], yr[3];
    for (int k = 0; k < 3; ++k) {
      px[k] = in.Xv[u][2 * k] - X[0];
      py[k] = in.Xv[u][2 * k + 1] - X[1];
      xr[k] = J[0] * px[k] + J[1] * py[k] - (1.0 / 3.0);
      yr[k] = J[2] * px[k] + J[3] * py[k] - (1.0 / 3.0);
    }
    double xrb[3] = {0, 0, 0}, yrb[3] = {0, 0, 0};
    tri_monomial_avgs_rev<M>(xr, yr, rb, xrb, yrb);
    for (int k = 0; k < 3; ++k) {
      const double pxb = J[0] * xrb[k] + J[2] * yrb[k], pyb = J[1] * xrb[k] + J[3] * yrb[k];
      pJ[0] += xrb[k] * px[k];
      pJ[1] += xrb[k] * py[k];
      pJ[2] += yrb[k] * px[k];
      pJ[3] += yrb[k] * py[k];
      Xvb[u][2 * k] += pxb;
      Xvb[u][2 * k + 1] += pyb;
      pX[0] -= pxb;
      pX[1] -= pyb;
    }
  }
  for (int k = 0; k < 4; ++k) pQ[k] = tm.sum(pQ[k]);
  for (int k = 0; k < 6; ++k) pX[k] = tm.sum(pX[k]);
  for (int k = 0; k < 4; ++k) pJ[k] = tm.sum(pJ[k]);
  if (tm.rank == 0) {
    // J = inverse of the element's affine map
    double jab = pJ[3] * tp.idet, jbb = -pJ[1] * tp.idet, jcb = -pJ[2] * tp.idet, jdb = pJ[0] * tp.idet;
    const double idb = pJ[0] * tp.jd - pJ[1] * tp.jb - pJ[2] * tp.jc + pJ[3] * tp.ja;
    const double detb = -idb * tp.idet * tp.idet;
    jab += detb * tp.jd; jdb += detb * tp.ja; jbb -= detb * tp.jc; jcb -= detb * tp.jb;
    pX[2] += jab; pX[0] -= jab;
    pX[4] += jbb; pX[0] -= jbb;
    pX[3] += jcb; pX[1] -= jcb;
    pX[5] += jdb; pX[1] -= jdb;
    for (int k = 0; k < 6; ++k) Xb[k] += pX[k];
    for (int v = 0; v < 4; ++v) Qb[v] += pQ[v];
  }
  tm.sync();
}

// ---------------------------------------------------------------------------
// Predictor of one element and its derived tables
// ---------------------------------------------------------------------------
constexpr int kMaxIt = 6;  // Picard iterations the reverse can store
// slots of a node's metric terms (node_geo)
enum { kGxx, kGxe, kGyx, kGye, kGxt, kGyt, kGid, kGxix, kGxiy, kGetx, kGety, kGxit, kGett, kNGeo };

template <int M>
struct PredTape {
  using S = Sz<M>;
  double q[kMaxIt][S::Nst][4];   // iterate entering iteration it
  double x[kMaxIt][S::Nst][2];
  double qf[S::Nst][4];          // final predictor
  int bad;                       // a non-physical node: the forward fell back to w_h
};

template <int M>
struct PredTables {
  using S = Sz<M>;
  double tr[3][S::Nt][S::Nt][4];  // edge, Gauss point, tau power, variable
  double av[S::Nt][4];
  double vd[6][S::Nt];            // vertex k, component c -> [2k + c], powers 1..Nt
};

// work arrays of the predictor (forward iterate, nodal fluxes, P and V) and
// of its reverse
template <int M>
struct PredWork {
  using S = Sz<M>;
  double q[S::Nst][4], x[S::Nst][2], F[S::Nst][4], G[S::Nst][4], P[S::Nst][4], V[S::Nst][2];
  double geo[S::Nst][kNGeo];
};
template <int M>
struct PredRev {
  using S = Sz<M>;
  double qb[S::Nst][4], xb[S::Nst][2], qo[S::Nst][4], xo[S::Nst][2], Pb[S::Nst][4], Vb[S::Nst][2];
  double F[S::Nst][4], G[S::Nst][4];
  // node-local adjoints of the derivative sums at each node: Q_xi, Q_eta,
  // f_xi, f_eta, g_xi, g_eta (4 each), x_xi, x_eta, y_xi, y_eta, x_tau, y_tau
  double dq[S::Nst][6][4], dx[S::Nst][6];
  double part[S::Nst][4][6];  // per variable: adjoints of xi_t, eta_t, xi_x, eta_x, xi_y, eta_y
  double fgq[S::Nst][3][4];   // per variable: gathered adjoints of q, f, g at a node
  double geo[S::Nst][kNGeo];  // metric terms of every node (node_geo)
};

// metric terms of node (t, s) of an iterate: x_xi, x_eta, y_xi, y_eta, x_tau,
// y_tau (per unit time), 1/det and the inverse map xi_x, xi_y, eta_x, eta_y,
// xi_t, eta_t, stored as geo[13] in that order (xx xe yx ye xt yt idet xix xiy
// etx ety xit ett)
template <int M>
AW_HD inline void node_geo(const Tab& T, const double (*x)[2], int t, int s, double idt, bool stat, double* g) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, Nt = S::Nt;
  double xx = 0.0, xe = 0.0, yx = 0.0, ye = 0.0;
  for (int r = 0; r < Mc; ++r) {
    const double a = T.Dxi[s][r], b = T.Deta[s][r];
    const int lr = t * Mc + r;
    xx += a * x[lr][0]; xe += b * x[lr][0];
    yx += a * x[lr][1]; ye += b * x[lr][1];
  }
  double xt = 0.0, yt = 0.0;
  if (!stat) {
    for (int u = 0; u < Nt; ++u) {
      xt += T.Dtau[t][u] * x[u * Mc + s][0];
      yt += T.Dtau[t][u] * x[u * Mc + s][1];
    }
    xt *= idt;
    yt *= idt;
  }
  const double idet = 1.0 / (xx * ye - xe * yx);
  const double xix = ye * idet, xiy = -xe * idet, etx = -yx * idet, ety = xx * idet;
  g[kGxx] = xx; g[kGxe] = xe; g[kGyx] = yx; g[kGye] = ye; g[kGxt] = xt; g[kGyt] = yt; g[kGid] = idet;
  g[kGxix] = xix; g[kGxiy] = xiy; g[kGetx] = etx; g[kGety] = ety;
  g[kGxit] = -(xix * xt + xiy * yt);
  g[kGett] = -(etx * xt + ety * yt);
}

// reference-space derivatives of variable v of q, f and g at node (t, s):
// d = {Q_xi, Q_eta, f_xi, f_eta, g_xi, g_eta}
template <int M>
AW_HD inline void node_sums_v(const Tab& T, const double (*q)[4], const double (*F)[4], const double (*G)[4], int t,
                              int s, int v, double* d) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc;
  double Qx = 0.0, Qe = 0.0, fx = 0.0, fe = 0.0, gx = 0.0, ge = 0.0;
  for (int r = 0; r < Mc; ++r) {
    const double a = T.Dxi[s][r], b = T.Deta[s][r];
    const int lr = t * Mc + r;
    Qx += a * q[lr][v]; Qe += b * q[lr][v];
    fx += a * F[lr][v]; fe += b * F[lr][v];
    gx += a * G[lr][v]; ge += b * G[lr][v];
  }
  d[0] = Qx; d[1] = Qe; d[2] = fx; d[3] = fe; d[4] = gx; d[5] = ge;
}

// first item of the per-node metric work in a loop that shares its pass with
// the Nst per-node items: the next warp boundary for a multi-warp team, so
// that the two kinds of work run on different warps
template <int M, class Tm>
AW_HD inline int geo_offset(const Tm& tm) {
  constexpr int Nst = Sz<M>::Nst;
  return tm.size >= 64 ? (Nst + 31) / 32 * 32 : Nst;
}

// Euler fluxes and mesh velocity of one node (one reciprocal of rho)
AW_HD inline void node_fluxes(const Tab& T, const double* q, double* f, double* g, double* V) {
  const double gm1 = T.gamma - 1.0;
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  f[0] = q[1]; f[1] = q[1] * u + p; f[2] = q[1] * v; f[3] = u * (q[3] + p);
  g[0] = q[2]; g[1] = q[2] * u; g[2] = q[2] * v + p; g[3] = v * (q[3] + p);
  if (V) {
    V[0] = T.eulerian ? 0.0 : u;
    V[1] = T.eulerian ? 0.0 : v;
  }
}

template <int M, class Tm>
AW_HD void pred_fwd(const Tab& T, int nit, const double (*w)[4], const double* X, double dts, PredTape<M>& tp,
                    PredTables<M>& out, PredWork<M>& wk, const Tm& tm) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, Nt = S::Nt, Nst = S::Nst;
  for (int l = tm.rank; l < Nst; l += tm.size) {
    const int s = l % Mc;
    for (int v = 0; v < 4; ++v) wk.q[l][v] = w[s][v];
    wk.x[l][0] = X[0] + (X[2] - X[0]) * T.lat[s][0] + (X[4] - X[0]) * T.lat[s][1];
    wk.x[l][1] = X[1] + (X[3] - X[1]) * T.lat[s][0] + (X[5] - X[1]) * T.lat[s][1];
  }
  tm.sync();
  const double idt = nit > 0 ? 1.0 / dts : 0.0;
  const int goff = geo_offset<M>(tm);
  for (int it = 0; it < nit; ++it) {
    const int nsl = it == 0 ? 1 : Nt;
    // per node: tape, fluxes; on other ranks: the node's metric terms
    for (int item = tm.rank; item < goff + nsl * Mc; item += tm.size) {
      if (item < Nst) {
        const int l = item;
        for (int v = 0; v < 4; ++v) tp.q[it][l][v] = wk.q[l][v];
        tp.x[it][l][0] = wk.x[l][0];
        tp.x[it][l][1] = wk.x[l][1];
        if (l < nsl * Mc) node_fluxes(T, wk.q[l], wk.F[l], wk.G[l], wk.V[l]);
      } else if (item >= goff) {
        const int l = item - goff;
        node_geo<M>(T, wk.x, l / Mc, l % Mc, idt, it == 0, wk.geo[l]);
      }
    }
    tm.sync();
    for (int it4 = tm.rank; it4 < nsl * Mc * 4; it4 += tm.size) {
      const int l = it4 / 4, v = it4 % 4;
      double d[6];
      node_sums_v<M>(T, tp.q[it], wk.F, wk.G, l / Mc, l % Mc, v, d);
      const double* g = wk.geo[l];
      const double fs = -(d[2] * g[kGxix] + d[3] * g[kGetx] + d[4] * g[kGxiy] + d[5] * g[kGety]);
      wk.P[l][v] = fs - (d[0] * g[kGxit] + d[1] * g[kGett]);
    }
    tm.sync();
    for (int l = Mc + tm.rank; l < Nst; l += tm.size) {
      const int t = l / Mc, s = l % Mc;
      for (int v = 0; v < 4; ++v) {
        double acc = 0.0;
        for (int u = 0; u < Nt; ++u) acc += T.B[t - 1][u] * wk.P[(it == 0 ? 0 : u) * Mc + s][v];
        wk.q[l][v] = tp.q[it][s][v] + dts * acc;
      }
      for (int c = 0; c < 2; ++c) {
        double acc = 0.0;
        for (int u = 0; u < Nt; ++u) acc += T.B[t - 1][u] * wk.V[(it == 0 ? 0 : u) * Mc + s][c];
        wk.x[l][c] = tp.x[it][s][c] + dts * acc;
      }
    }
    tm.sync();
  }
  const double gm1 = T.gamma - 1.0;
  int bad = 0;
  for (int l = tm.rank; l < Nst; l += tm.size) {
    if (!(wk.q[l][0] > 0.0) || !(pressure_of(gm1, wk.q[l]) > 0.0)) bad = 1;
    for (int v = 0; v < 4; ++v) tp.qf[l][v] = wk.q[l][v];
  }
  bad = tm.any(bad);
  if (tm.rank == 0) tp.bad = bad;
  tm.sync();
  // derived tables
  constexpr int nTr = 3 * Nt * 4, nItems = nTr + 4 + 6;
  for (int item = tm.rank; item < nItems; item += tm.size) {
    if (item < nTr) {
      const int e = item / (Nt * 4), g = (item / 4) % Nt, v = item % 4;
      double val[Nt];
      for (int tt = 0; tt < Nt; ++tt) {
        double acc = 0.0;
        for (int r = 0; r < Mc; ++r) acc += T.Tr[e][g][r] * tp.qf[tt * Mc + r][v];
        val[tt] = acc;
      }
      for (int p = 0; p < Nt; ++p) {
        double acc = 0.0;
        for (int tt = 0; tt < Nt; ++tt) acc += T.VtInv[p][tt] * val[tt];
        out.tr[e][g][p][v] = acc;
      }
    } else if (item < nTr + 4) {
      const int v = item - nTr;
      double val[Nt];
      for (int tt = 0; tt < Nt; ++tt) {
        double acc = 0.0;
        for (int r = 0; r < Mc; ++r) acc += T.wavg[r] * tp.qf[tt * Mc + r][v];
        val[tt] = acc;
      }
      for (int p = 0; p < Nt; ++p) {
        double acc = 0.0;
        for (int tt = 0; tt < Nt; ++tt) acc += T.VtInv[p][tt] * val[tt];
        out.av[p][v] = acc;
      }
    } else {
      const int kc = item - nTr - 4, k = kc / 2, c = kc % 2, sn = T.vnode[k];
      double vel[Nt];
      for (int tt = 0; tt < Nt; ++tt) {
        const double* qq = tp.qf[tt * Mc + sn];
        vel[tt] = T.eulerian ? 0.0 : qq[1 + c] / qq[0];
      }
      for (int p = 0; p < Nt; ++p) {
        double acc = 0.0;
        for (int tt = 0; tt < Nt; ++tt) acc += T.VtInv[p][tt] * vel[tt];
        out.vd[kc][p] = acc / (p + 1);
      }
    }
  }
  tm.sync();
}

// Reverse of pred_fwd: tb = dJ/d(tables); adds to wb (Mc x 4, each node by
// one rank) and Xb (6, rank 0).  Every reverse sum is a gather: each node's
// adjoint is written by one rank only.
template <int M, class Tm>
AW_HD void pred_rev(const Tab& T, int nit, double dts, const PredTape<M>& tp, const PredTables<M>& tb,
                    double (*wb)[4], double* Xb, PredRev<M>& wk, const Tm& tm) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, Nt = S::Nt, Nst = S::Nst;
  // tables: the adjoint of every node of the final predictor (per variable,
  // then the vertex velocities per node).  First the tables' adjoints through
  // the tau powers, once per (edge, Gauss point, time slice, variable) and per
  // (time slice, variable) of the average, not once per node; then per node.
  double* vb = &wk.dq[0][0][0];  // free until the Picard iterations' reverse
  constexpr int nV = 3 * Nt * Nt * 4, nA = Nt * 4;
  static_assert(nV + nA <= Nst * 6 * 4, "table adjoints exceed their scratch");
  for (int it = tm.rank; it < nV + nA; it += tm.size) {
    double acc = 0.0;
    if (it < nV) {
      const int e = it / (Nt * Nt * 4), g = (it / (Nt * 4)) % Nt, tt = (it / 4) % Nt, v = it % 4;
      for (int p = 0; p < Nt; ++p) acc += T.VtInv[p][tt] * tb.tr[e][g][p][v];
    } else {
      const int tt = (it - nV) / 4, v = (it - nV) % 4;
      for (int p = 0; p < Nt; ++p) acc += T.VtInv[p][tt] * tb.av[p][v];
    }
    vb[it] = acc;
  }
  tm.sync();
  for (int it4 = tm.rank; it4 < Nst * 4; it4 += tm.size) {
    const int l = it4 / 4, v = it4 % 4, tt = l / Mc, r = l % Mc;
    double acc = 0.0;
    for (int e = 0; e < 3; ++e)
      for (int g = 0; g < Nt; ++g) acc += T.Tr[e][g][r] * vb[((e * Nt + g) * Nt + tt) * 4 + v];
    acc += T.wavg[r] * vb[nV + tt * 4 + v];
    wk.qb[l][v] = acc;
  }
  tm.sync();
  for (int l = tm.rank; l < Nst; l += tm.size) {
    const int tt = l / Mc, r = l % Mc;
    if (!T.eulerian)
      for (int k = 0; k < 3; ++k) {
        if (T.vnode[k] != r) continue;
        const double* qq = tp.qf[l];
        const double ir = 1.0 / qq[0];
        for (int c = 0; c < 2; ++c) {
          double velb = 0.0;
          for (int p = 0; p < Nt; ++p) velb += T.VtInv[p][tt] * tb.vd[2 * k + c][p] / (p + 1);
          wk.qb[l][1 + c] += velb * ir;
          wk.qb[l][0] -= velb * qq[1 + c] * ir * ir;
        }
      }
    wk.xb[l][0] = wk.xb[l][1] = 0.0;
  }
  tm.sync();
  // Picard iterations in reverse
  const double idt = nit > 0 ? 1.0 / dts : 0.0;
  const int goff = geo_offset<M>(tm);
  for (int it = nit - 1; it >= 0; --it) {
    const int nsl = it == 0 ? 1 : Nt;
    const bool stat = it == 0;
    for (int item = tm.rank; item < goff + nsl * Mc; item += tm.size) {
      if (item >= goff) {  // the node's metric terms in the iterate
        const int l = item - goff;
        node_geo<M>(T, tp.x[it], l / Mc, l % Mc, idt, stat, wk.geo[l]);
        continue;
      }
      if (item >= Nst) continue;
      const int l = item;
      const int u = l / Mc, s = l % Mc;
      double P[4] = {0, 0, 0, 0}, V[2] = {0, 0};
      if (it > 0 || u == 0)
        for (int t = 1; t < Nt; ++t) {
          double bt = 0.0;
          if (it > 0) bt = T.B[t - 1][u];
          else
            for (int uu = 0; uu < Nt; ++uu) bt += T.B[t - 1][uu];
          for (int v = 0; v < 4; ++v) P[v] += dts * bt * wk.qb[t * Mc + s][v];
          for (int c = 0; c < 2; ++c) V[c] += dts * bt * wk.xb[t * Mc + s][c];
        }
      for (int v = 0; v < 4; ++v) wk.Pb[l][v] = P[v];
      wk.Vb[l][0] = V[0];
      wk.Vb[l][1] = V[1];
      if (u == 0) {
        for (int v = 0; v < 4; ++v) {
          double acc = wk.qb[s][v];
          for (int t = 1; t < Nt; ++t) acc += wk.qb[t * Mc + s][v];
          wk.qo[l][v] = acc;
        }
        for (int c = 0; c < 2; ++c) {
          double acc = wk.xb[s][c];
          for (int t = 1; t < Nt; ++t) acc += wk.xb[t * Mc + s][c];
          wk.xo[l][c] = acc;
        }
      } else {
        for (int v = 0; v < 4; ++v) wk.qo[l][v] = 0.0;
        wk.xo[l][0] = wk.xo[l][1] = 0.0;
      }
      if (l < nsl * Mc) node_fluxes(T, tp.q[it][l], wk.F[l], wk.G[l], nullptr);
    }
    tm.sync();
    // node-local reverse of P at every node that computed one: per variable,
    // then the metric terms of the node
    for (int it4 = tm.rank; it4 < nsl * Mc * 4; it4 += tm.size) {
      const int l = it4 / 4, v = it4 % 4;
      double d[6];
      node_sums_v<M>(T, tp.q[it], wk.F, wk.G, l / Mc, l % Mc, v, d);
      const double* g = wk.geo[l];
      const double Pb = wk.Pb[l][v];
      wk.dq[l][0][v] = -Pb * g[kGxit]; wk.dq[l][1][v] = -Pb * g[kGett];
      wk.dq[l][2][v] = -Pb * g[kGxix]; wk.dq[l][3][v] = -Pb * g[kGetx];
      wk.dq[l][4][v] = -Pb * g[kGxiy]; wk.dq[l][5][v] = -Pb * g[kGety];
      double* pt = wk.part[l][v];
      pt[0] = -Pb * d[0]; pt[1] = -Pb * d[1];
      pt[2] = -Pb * d[2]; pt[3] = -Pb * d[3]; pt[4] = -Pb * d[4]; pt[5] = -Pb * d[5];
    }
    tm.sync();
    for (int l = tm.rank; l < nsl * Mc; l += tm.size) {
      struct {
        double xx, xe, yx, ye, xt, yt, idet, xix, xiy, etx, ety, xit, ett;
      } n;
      const double* g = wk.geo[l];
      n.xx = g[kGxx]; n.xe = g[kGxe]; n.yx = g[kGyx]; n.ye = g[kGye]; n.xt = g[kGxt]; n.yt = g[kGyt];
      n.idet = g[kGid]; n.xix = g[kGxix]; n.xiy = g[kGxiy]; n.etx = g[kGetx]; n.ety = g[kGety];
      n.xit = g[kGxit]; n.ett = g[kGett];
      double xitb = 0, ettb = 0, xixb = 0, etxb = 0, xiyb = 0, etyb = 0;
      for (int v = 0; v < 4; ++v) {
        const double* pt = wk.part[l][v];
        xitb += pt[0]; ettb += pt[1]; xixb += pt[2]; etxb += pt[3]; xiyb += pt[4]; etyb += pt[5];
      }
      double xtb = 0, ytb = 0;
      xixb -= xitb * n.xt; xiyb -= xitb * n.yt; xtb -= xitb * n.xix; ytb -= xitb * n.xiy;
      etxb -= ettb * n.xt; etyb -= ettb * n.yt; xtb -= ettb * n.etx; ytb -= ettb * n.ety;
      double xxb = 0, xeb = 0, yxb = 0, yeb = 0, idb = 0;
      yeb += xixb * n.idet; idb += xixb * n.ye;
      xeb -= xiyb * n.idet; idb -= xiyb * n.xe;
      yxb -= etxb * n.idet; idb -= etxb * n.yx;
      xxb += etyb * n.idet; idb += etyb * n.xx;
      const double detb = -idb * n.idet * n.idet;
      xxb += detb * n.ye; yeb += detb * n.xx; xeb -= detb * n.yx; yxb -= detb * n.xe;
      wk.dx[l][0] = xxb; wk.dx[l][1] = xeb; wk.dx[l][2] = yxb; wk.dx[l][3] = yeb;
      wk.dx[l][4] = stat ? 0.0 : xtb;
      wk.dx[l][5] = stat ? 0.0 : ytb;
    }
    tm.sync();
    // gather onto every node of the iterate: per variable, then per node
    for (int it4 = tm.rank; it4 < nsl * Mc * 4; it4 += tm.size) {
      const int l = it4 / 4, v = it4 % 4;
      const int t = l / Mc, r = l % Mc;
      double qa = 0.0, fb = 0.0, gb = 0.0;
      for (int s = 0; s < Mc; ++s) {
        const double a = T.Dxi[s][r], b = T.Deta[s][r];
        const int ls = t * Mc + s;
        qa += a * wk.dq[ls][0][v] + b * wk.dq[ls][1][v];
        fb += a * wk.dq[ls][2][v] + b * wk.dq[ls][3][v];
        gb += a * wk.dq[ls][4][v] + b * wk.dq[ls][5][v];
      }
      wk.fgq[l][0][v] = qa;
      wk.fgq[l][1][v] = fb;
      wk.fgq[l][2][v] = gb;
    }
    tm.sync();
    for (int l = tm.rank; l < nsl * Mc; l += tm.size) {
      const int t = l / Mc, r = l % Mc;
      double qa[4], x0 = 0.0, x1 = 0.0;
      for (int v = 0; v < 4; ++v) qa[v] = wk.fgq[l][0][v];
      for (int s = 0; s < Mc; ++s) {
        const double a = T.Dxi[s][r], b = T.Deta[s][r];
        const int ls = t * Mc + s;
        x0 += a * wk.dx[ls][0] + b * wk.dx[ls][1];
        x1 += a * wk.dx[ls][2] + b * wk.dx[ls][3];
      }
      if (!stat)
        for (int tt = 0; tt < Nt; ++tt) {
          x0 += idt * T.Dtau[tt][t] * wk.dx[tt * Mc + r][4];
          x1 += idt * T.Dtau[tt][t] * wk.dx[tt * Mc + r][5];
        }
      const double* q = tp.q[it][l];
      euler_fg_rev(T.gamma - 1.0, q, wk.fgq[l][1], wk.fgq[l][2], qa);
      if (!T.eulerian) {
        const double ir = 1.0 / q[0];
        qa[1] += wk.Vb[l][0] * ir;
        qa[2] += wk.Vb[l][1] * ir;
        qa[0] -= (wk.Vb[l][0] * q[1] + wk.Vb[l][1] * q[2]) * ir * ir;
      }
      for (int v = 0; v < 4; ++v) wk.qo[l][v] += qa[v];
      wk.xo[l][0] += x0;
      wk.xo[l][1] += x1;
    }
    tm.sync();
    for (int l = tm.rank; l < Nst; l += tm.size) {
      for (int v = 0; v < 4; ++v) wk.qb[l][v] = wk.qo[l][v];
      wk.xb[l][0] = wk.xo[l][0];
      wk.xb[l][1] = wk.xo[l][1];
    }
    tm.sync();
  }
  // initial iterate: q = w on every slice, x = lattice positions
  double pX[6] = {0, 0, 0, 0, 0, 0};
  for (int s = tm.rank; s < Mc; s += tm.size) {
    double x0b = 0.0, x1b = 0.0;
    for (int t = 0; t < Nt; ++t) {
      for (int v = 0; v < 4; ++v) wb[s][v] += wk.qb[t * Mc + s][v];
      x0b += wk.xb[t * Mc + s][0];
      x1b += wk.xb[t * Mc + s][1];
    }
    const double l0 = T.lat[s][0], l1 = T.lat[s][1];
    pX[0] += x0b * (1.0 - l0 - l1); pX[2] += x0b * l0; pX[4] += x0b * l1;
    pX[1] += x1b * (1.0 - l0 - l1); pX[3] += x1b * l0; pX[5] += x1b * l1;
  }
  for (int k = 0; k < 6; ++k) pX[k] = tm.sum(pX[k]);
  if (tm.rank == 0)
    for (int k = 0; k < 6; ++k) Xb[k] += pX[k];
  tm.sync();
}

// ---------------------------------------------------------------------------
// One swept edge surface
// ---------------------------------------------------------------------------
template <int M>
struct EdgeIn {
  using S = Sz<M>;
  double P[4][2];                 // old a, old b, new b, new a (periodic shift applied)
  double tk[4];                   // their ticks
  double tsec;                    // seconds per tick
  double trL[S::Nt][S::Nt][4];    // left trace: Gauss point, tau power, variable
  double trR[S::Nt][S::Nt][4];    // right trace, its own Gauss point order
  double tL, dtL, tR, dtR;        // ticks of the two sides
  double qg[4];                   // transmissive outer state: the left element's average
  int has_R, bc;                  // bc 0 wall, 1 transmissive (no right side)
};

AW_HD inline void rusanov_fwd(double g, const double* qm, const double* qp, const double* n, double* F) {
  const double rim = 1.0 / qm[0], rip = 1.0 / qp[0];
  const double um = qm[1] * rim, vm = qm[2] * rim, up = qp[1] * rip, vp = qp[2] * rip;
  const double pm = (g - 1.0) * (qm[3] - 0.5 * (qm[1] * um + qm[2] * vm));
  const double pp = (g - 1.0) * (qp[3] - 0.5 * (qp[1] * up + qp[2] * vp));
  const double nn2 = n[0] * n[0] + n[1] * n[1];
  const double cmn = sqrt(g * pm * rim * nn2), cpn = sqrt(g * pp * rip * nn2);
  const double wm = um * n[0] + vm * n[1] + n[2], wp = up * n[0] + vp * n[1] + n[2];
  const double sm = fabs(wm) + cmn, sp = fabs(wp) + cpn;
  const double smax = fmax(sm, sp);
  const double vnm = um * n[0] + vm * n[1], vnp = up * n[0] + vp * n[1];
  const double Fm[4] = {qm[0] * wm, qm[1] * wm + pm * n[0], qm[2] * wm + pm * n[1], qm[3] * wm + pm * vnm};
  const double Fp[4] = {qp[0] * wp, qp[1] * wp + pp * n[0], qp[2] * wp + pp * n[1], qp[3] * wp + pp * vnp};
  for (int v = 0; v < 4; ++v) F[v] = 0.5 * (Fm[v] + Fp[v]) - 0.5 * smax * (qp[v] - qm[v]);
}

// one side's contribution F_side(q) = q w + p (0, n0, n1, vn), w = v.n + n2;
// adds its reverse to qb, nb
AW_HD inline void side_flux_rev(double g, const double* q, const double* n, const double* Fb, double* qb, double* nb) {
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = (g - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  const double w = u * n[0] + v * n[1] + n[2], vn = u * n[0] + v * n[1];
  double wb = 0.0, pb = 0.0, vnb = 0.0;
  for (int k = 0; k < 4; ++k) {
    qb[k] += Fb[k] * w;
    wb += Fb[k] * q[k];
  }
  pb += Fb[1] * n[0] + Fb[2] * n[1] + Fb[3] * vn;
  nb[0] += Fb[1] * p;
  nb[1] += Fb[2] * p;
  vnb += Fb[3] * p;
  double ub = wb * n[0] + vnb * n[0], vb = wb * n[1] + vnb * n[1];
  nb[0] += (wb + vnb) * u;
  nb[1] += (wb + vnb) * v;
  nb[2] += wb;
  // p = (g-1)(E - (q1 u + q2 v)/2)
  qb[3] += pb * (g - 1.0);
  qb[1] -= 0.5 * (g - 1.0) * pb * u;
  qb[2] -= 0.5 * (g - 1.0) * pb * v;
  ub -= 0.5 * (g - 1.0) * pb * q[1];
  vb -= 0.5 * (g - 1.0) * pb * q[2];
  qb[1] += ub * ir;
  qb[2] += vb * ir;
  qb[0] -= (ub * q[1] + vb * q[2]) * ir * ir;
}

// wave-speed bound s = |v.n + n2| + sqrt(g p / rho * |n_xy|^2); reverse adds sb ds
AW_HD inline double speed_of(double g, const double* q, const double* n) {
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = (g - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  const double nn2 = n[0] * n[0] + n[1] * n[1];
  return fabs(u * n[0] + v * n[1] + n[2]) + sqrt(g * p * ir * nn2);
}
AW_HD inline void speed_rev(double g, const double* q, const double* n, double sb, double* qb, double* nb) {
  const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
  const double p = (g - 1.0) * (q[3] - 0.5 * (q[1] * u + q[2] * v));
  const double nn2 = n[0] * n[0] + n[1] * n[1];
  const double w = u * n[0] + v * n[1] + n[2];
  const double cn = sqrt(g * p * ir * nn2);
  const double wb = w >= 0.0 ? sb : -sb;
  double ub = wb * n[0], vb = wb * n[1];
  nb[0] += wb * u;
  nb[1] += wb * v;
  nb[2] += wb;
  if (cn > 0.0) {
    const double zb = sb / (2.0 * cn);  // z = g p ir nn2
    const double pb = zb * g * ir * nn2;
    const double irb = zb * g * p * nn2;
    const double nn2b = zb * g * p * ir;
    nb[0] += 2.0 * n[0] * nn2b;
    nb[1] += 2.0 * n[1] * nn2b;
    qb[3] += pb * (g - 1.0);
    qb[1] -= 0.5 * (g - 1.0) * pb * u;
    qb[2] -= 0.5 * (g - 1.0) * pb * v;
    ub -= 0.5 * (g - 1.0) * pb * q[1];
    vb -= 0.5 * (g - 1.0) * pb * q[2];
    qb[0] -= irb * ir * ir;
  }
  qb[1] += ub * ir;
  qb[2] += vb * ir;
  qb[0] -= (ub * q[1] + vb * q[2]) * ir * ir;
}

template <int M>
AW_HD inline void edge_point(const Tab& T, const EdgeIn<M>& in, int gx, int gt, double* qm, double* qp, double* n,
                             double* dchi, double* dtau, double* tl, double* tr) {
  constexpr int Nt = Sz<M>::Nt;
  const double chi = T.glx[gx], tau = T.glx[gt];
  double P[4][3];
  for (int k = 0; k < 4; ++k) {
    P[k][0] = in.P[k][0];
    P[k][1] = in.P[k][1];
    P[k][2] = in.tk[k] * in.tsec;
  }
  for (int c = 0; c < 3; ++c) {
    dchi[c] = (1.0 - tau) * (P[1][c] - P[0][c]) + tau * (P[2][c] - P[3][c]);
    dtau[c] = (1.0 - chi) * (P[3][c] - P[0][c]) + chi * (P[2][c] - P[1][c]);
  }
  n[0] = dchi[1] * dtau[2] - dchi[2] * dtau[1];
  n[1] = dchi[2] * dtau[0] - dchi[0] * dtau[2];
  n[2] = dchi[0] * dtau[1] - dchi[1] * dtau[0];
  const double tt = (1 - chi) * (1 - tau) * in.tk[0] + chi * (1 - tau) * in.tk[1] + chi * tau * in.tk[2] +
                    (1 - chi) * tau * in.tk[3];
  *tl = in.dtL > 0 ? (tt - in.tL) / in.dtL : 0.0;
  for (int v = 0; v < 4; ++v) {
    double acc = in.trL[gx][Nt - 1][v];
    for (int p = Nt - 2; p >= 0; --p) acc = acc * *tl + in.trL[gx][p][v];
    qm[v] = acc;
  }
  *tr = 0.0;
  if (in.has_R) {
    *tr = in.dtR > 0 ? (tt - in.tR) / in.dtR : 0.0;
    for (int v = 0; v < 4; ++v) {
      double acc = in.trR[Nt - 1 - gx][Nt - 1][v];
      for (int p = Nt - 2; p >= 0; --p) acc = acc * *tr + in.trR[Nt - 1 - gx][p][v];
      qp[v] = acc;
    }
  } else if (in.bc == 1) {
    for (int v = 0; v < 4; ++v) qp[v] = in.qg[v];
  } else {
    for (int v = 0; v < 4; ++v) qp[v] = qm[v];
    if (in.bc == 0) {
      const double nn = n[0] * n[0] + n[1] * n[1];
      if (nn > 0.0) {
        const double mn = (qm[1] * n[0] + qm[2] * n[1]) / nn;
        qp[1] = qm[1] - 2.0 * mn * n[0];
        qp[2] = qm[2] - 2.0 * mn * n[1];
      }
    }
  }
}

template <int M>
AW_HD void edge_fwd(const Tab& T, const EdgeIn<M>& in, double* G) {
  constexpr int Nt = Sz<M>::Nt;
  for (int v = 0; v < 4; ++v) G[v] = 0.0;
  for (int gx = 0; gx < Nt; ++gx)
    for (int gt = 0; gt < Nt; ++gt) {
      double qm[4], qp[4], n[3], dchi[3], dtau[3], tl, tr, F[4];
      edge_point<M>(T, in, gx, gt, qm, qp, n, dchi, dtau, &tl, &tr);
      rusanov_fwd(T.gamma, qm, qp, n, F);
      const double wq = T.glw[gx] * T.glw[gt];
      for (int v = 0; v < 4; ++v) G[v] += wq * F[v];
    }
}

// reverse of the Gauss point (gx, gt) of edge_fwd: adds to Pb[4][2], the
// two traces' adjoints (row gx of the left trace, row Nt-1-gx of the right)
// and, on a transmissive edge, the outer state's adjoint qgb[4]
template <int M>
AW_HD void edge_point_rev(const Tab& T, const EdgeIn<M>& in, int gx, int gt, const double* Gb, double (*Pb)[2],
                          double (*trLb)[Sz<M>::Nt][4], double (*trRb)[Sz<M>::Nt][4], double* qgb) {
  constexpr int Nt = Sz<M>::Nt;
  const double g = T.gamma;
  double qm[4], qp[4], n[3], dchi[3], dtau[3], tl, tr;
  edge_point<M>(T, in, gx, gt, qm, qp, n, dchi, dtau, &tl, &tr);
  const double wq = T.glw[gx] * T.glw[gt];
  double Fb[4];
  for (int v = 0; v < 4; ++v) Fb[v] = wq * Gb[v];
  double qmb[4] = {0, 0, 0, 0}, qpb[4] = {0, 0, 0, 0}, nb[3] = {0, 0, 0};
  // F = (Fm + Fp)/2 - smax (qp - qm)/2
  const double sm = speed_of(g, qm, n), sp = speed_of(g, qp, n), smax = fmax(sm, sp);
  double half[4], smaxb = 0.0;
  for (int v = 0; v < 4; ++v) {
    half[v] = 0.5 * Fb[v];
    smaxb -= 0.5 * Fb[v] * (qp[v] - qm[v]);
    qpb[v] -= 0.5 * smax * Fb[v];
    qmb[v] += 0.5 * smax * Fb[v];
  }
  side_flux_rev(g, qm, n, half, qmb, nb);
  side_flux_rev(g, qp, n, half, qpb, nb);
  if (sm >= sp) speed_rev(g, qm, n, smaxb, qmb, nb);
  else speed_rev(g, qp, n, smaxb, qpb, nb);
  // right state
  if (in.has_R) {
    double tp_ = 1.0;
    for (int p = 0; p < Nt; ++p) {
      for (int v = 0; v < 4; ++v) trRb[Nt - 1 - gx][p][v] += qpb[v] * tp_;
      tp_ *= tr;
    }
  } else if (in.bc == 1) {
    for (int v = 0; v < 4; ++v) qgb[v] += qpb[v];
  } else {
    for (int v = 0; v < 4; ++v) qmb[v] += (v == 1 || v == 2) ? 0.0 : qpb[v];
    const double nn = n[0] * n[0] + n[1] * n[1];
    if (in.bc == 0 && nn > 0.0) {
      const double mn = (qm[1] * n[0] + qm[2] * n[1]) / nn;
      qmb[1] += qpb[1];
      qmb[2] += qpb[2];
      const double mnb = -2.0 * (qpb[1] * n[0] + qpb[2] * n[1]);
      nb[0] -= 2.0 * mn * qpb[1];
      nb[1] -= 2.0 * mn * qpb[2];
      qmb[1] += mnb * n[0] / nn;
      qmb[2] += mnb * n[1] / nn;
      nb[0] += mnb * qm[1] / nn;
      nb[1] += mnb * qm[2] / nn;
      const double nnb = -mnb * mn / nn;
      nb[0] += 2.0 * n[0] * nnb;
      nb[1] += 2.0 * n[1] * nnb;
    } else {
      qmb[1] += qpb[1];
      qmb[2] += qpb[2];
    }
  }
  {
    double tp_ = 1.0;
    for (int p = 0; p < Nt; ++p) {
      for (int v = 0; v < 4; ++v) trLb[gx][p][v] += qmb[v] * tp_;
      tp_ *= tl;
    }
  }
  // n = dchi x dtau (spatial components of the corners only)
  double dchib[3], dtaub[3];
  dchib[0] = dtau[1] * nb[2] - dtau[2] * nb[1];
  dchib[1] = dtau[2] * nb[0] - dtau[0] * nb[2];
  dchib[2] = dtau[0] * nb[1] - dtau[1] * nb[0];
  dtaub[0] = nb[1] * dchi[2] - nb[2] * dchi[1];
  dtaub[1] = nb[2] * dchi[0] - nb[0] * dchi[2];
  dtaub[2] = nb[0] * dchi[1] - nb[1] * dchi[0];
  const double chi = T.glx[gx], tau = T.glx[gt];
  for (int c = 0; c < 2; ++c) {
    Pb[1][c] += (1.0 - tau) * dchib[c]; Pb[0][c] -= (1.0 - tau) * dchib[c];
    Pb[2][c] += tau * dchib[c]; Pb[3][c] -= tau * dchib[c];
    Pb[3][c] += (1.0 - chi) * dtaub[c]; Pb[0][c] -= (1.0 - chi) * dtaub[c];
    Pb[2][c] += chi * dtaub[c]; Pb[1][c] -= chi * dtaub[c];
  }
}

// reverse of edge_fwd: adds to Pb[4][2] and the two traces' adjoints
template <int M>
AW_HD void edge_rev(const Tab& T, const EdgeIn<M>& in, const double* Gb, double (*Pb)[2], double (*trLb)[Sz<M>::Nt][4],
                    double (*trRb)[Sz<M>::Nt][4], double* qgb) {
  constexpr int Nt = Sz<M>::Nt;
  for (int gx = 0; gx < Nt; ++gx)
    for (int gt = 0; gt < Nt; ++gt) edge_point_rev<M>(T, in, gx, gt, Gb, Pb, trLb, trRb, qgb);
}

// ---------------------------------------------------------------------------
// Node solver for one node: mass-weighted mean of the Voronoi elements'
// time-integrated vertex velocities over [tau0, tau1] of each element
// ---------------------------------------------------------------------------
template <int M>
struct NodeElem {
  double rho, X[6];       // element average density and vertices (sweep start)
  double vd[2][Sz<M>::Nt];// vertex displacement coefficients of this node, x and y
  double tau0, tau1, dts; // dts = 0: the element has finished (no motion)
};

template <int M>
AW_HD inline void node_elem_disp(const NodeElem<M>& e, double* D) {
  constexpr int Nt = Sz<M>::Nt;
  D[0] = D[1] = 0.0;
  if (!(e.dts > 0.0)) return;
  for (int c = 0; c < 2; ++c) {
    double a0 = e.vd[c][Nt - 1], a1 = e.vd[c][Nt - 1];
    for (int p = Nt - 2; p >= 0; --p) {
      a0 = a0 * e.tau0 + e.vd[c][p];
      a1 = a1 * e.tau1 + e.vd[c][p];
    }
    D[c] = e.dts * (a1 * e.tau1 - a0 * e.tau0);
  }
}

template <int M>
AW_HD void node_fwd(int nv, const NodeElem<M>* el, int type, const double* nrm, double* D) {
  double num0 = 0.0, num1 = 0.0, den = 0.0;
  for (int k = 0; k < nv; ++k) {
    const double mu = el[k].rho * tri_area(el[k].X);
    double Dk[2];
    node_elem_disp<M>(el[k], Dk);
    num0 += mu * Dk[0];
    num1 += mu * Dk[1];
    den += mu;
  }
  D[0] = num0 / den;
  D[1] = num1 / den;
  if (type == 1) {
    const double dn = D[0] * nrm[0] + D[1] * nrm[1];
    D[0] -= dn * nrm[0];
    D[1] -= dn * nrm[1];
  } else if (type == 2) {
    D[0] = D[1] = 0.0;
  }
}

// reverse: Db = dJ/dD; adds to rhob[k], Xb[k][6], vdb[k][2][Nt]
template <int M>
AW_HD void node_rev(int nv, const NodeElem<M>* el, int type, const double* nrm, const double* Db_in, double* rhob,
                    double (*Xb)[6], double (*vdb)[2][Sz<M>::Nt]) {
  constexpr int Nt = Sz<M>::Nt;
  double Db[2] = {Db_in[0], Db_in[1]};
  if (type == 1) {
    const double dn = Db[0] * nrm[0] + Db[1] * nrm[1];
    Db[0] -= dn * nrm[0];
    Db[1] -= dn * nrm[1];
  } else if (type == 2) {
    return;
  }
  double num0 = 0.0, num1 = 0.0, den = 0.0;
  for (int k = 0; k < nv; ++k) {
    const double mu = el[k].rho * tri_area(el[k].X);
    double Dk[2];
    node_elem_disp<M>(el[k], Dk);
    num0 += mu * Dk[0];
    num1 += mu * Dk[1];
    den += mu;
  }
  const double D0 = num0 / den, D1 = num1 / den;
  const double n0b = Db[0] / den, n1b = Db[1] / den, denb = -(Db[0] * D0 + Db[1] * D1) / den;
  for (int k = 0; k < nv; ++k) {
    const double area = tri_area(el[k].X), mu = el[k].rho * area;
    double Dk[2];
    node_elem_disp<M>(el[k], Dk);
    const double mub = n0b * Dk[0] + n1b * Dk[1] + denb;
    rhob[k] += mub * area;
    tri_area_rev(el[k].X, mub * el[k].rho, Xb[k]);
    if (el[k].dts > 0.0) {
      const double Dkb[2] = {n0b * mu, n1b * mu};
      double p1 = el[k].tau1, p0 = el[k].tau0;
      for (int p = 0; p < Nt; ++p) {
        // D = dts (sum_p vd[p] tau1^(p+1) - sum_p vd[p] tau0^(p+1))
        for (int c = 0; c < 2; ++c) vdb[k][c][p] += Dkb[c] * el[k].dts * (p1 - p0);
        p1 *= el[k].tau1;
        p0 *= el[k].tau0;
      }
    }
  }
}

}  // namespace adj
}  // namespace aw
