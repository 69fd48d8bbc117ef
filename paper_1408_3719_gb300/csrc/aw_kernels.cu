// Kernels of one LTS sweep (Sec. 2.6) on sm_103a, all FP64, launched in this
// order (one captured CUDA graph per sweep; k_nodes_grp and k_edges are two
// parallel branches of it):
//   k_ready        update criterion on S^W (eq. WENOupdate) for the candidate
//                  elements; compaction of the ready elements and their nodes
//   k_nodes_grp    node solver NS_cs (eqs. eqnNScs, NodesVel, newVertex)
//   k_edges        edges with a moved endpoint and the elements they touch
//   k_flux_grp     space-time fluxes through the swept edge surfaces (eqs.
//                  spacetimenodes, rusanov, STint) and their GCL normals
//   k_update       one-step FV update / memory variables (eqs. PDEfinal, Qm2, gcl)
//   k_recon_coop   virtual projection + WENO + local time step (eqs. virtGeom,
//                  virtCellaverage, intConsRec, weno, timestep)
//   k_predict_coop space-time Galerkin predictor (eqs. PDECG, pdef, CGfinal,
//                  newVertPos) and its derived tables (edge traces, averages,
//                  vertex displacement polynomials)
//   k_finish       commit the moved nodes, list the next sweep's candidates,
//                  reset the per-sweep counters
// Work lists are compacted with atomics on warp-aggregated slots (the ready
// list and the moved nodes by warp ballot); every
// per-element and per-node sum runs in a fixed order, so results do not
// depend on the order of the lists.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdio>

#include "aw_internal.h"

namespace aw {

namespace {

constexpr int kBlock = 128;

__device__ __forceinline__ double area6(const double* X) {
  return 0.5 * ((X[2] - X[0]) * (X[5] - X[1]) - (X[3] - X[1]) * (X[4] - X[0]));
}

__device__ __forceinline__ void set_error(Counters* cnt, int code, int elem) {
  if (atomicCAS(&cnt->err_code, 0, code) == 0) cnt->err_elem = elem;
}

__device__ __forceinline__ double pressure(const Tab& T, const double* q) {
  return (T.gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

// ---------------------------------------------------------------------------
// Candidates: every element in the first sweep after a state is loaded;
// afterwards the total stencils of the previous sweep's ready elements (the
// criterion of any other element reads only unchanged times).
__global__ void k_ready(Tab T, Dev d) {
  // eight lanes per candidate element, four candidates per warp; each lane
  // loads its UN total-stencil entries of a chunk (and their ticks) before
  // any of them is tested, and a chunk that finds a violation ends the test.
  // Compaction: a warp ballot of its ready candidates and of their new
  // vertices, one atomic per warp for each list, slots from the ballot's
  // prefix counts.
  constexpr int GL = 8, UN = 4;
  const int epoch = d.cnt->epoch;
  const long long Ts = d.cnt->t_sync;
  const int par = epoch & 1;
  const bool listed = d.cnt->cand_valid != 0 && !T.gts;
  const int n_items = listed ? d.cnt->n_cand[par] : d.ne;
  const int* clist = d.cand_list + (size_t)par * d.ne;
  const int lane = threadIdx.x & 31, gl = lane & (GL - 1);
  const unsigned gmask = 0xFFu << (lane & ~(GL - 1));
  const unsigned lt = (1u << lane) - 1u;  // lanes below this one
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) d.cnt->gts_min = LLONG_MAX;
  for (int qb = warp * (32 / GL); qb < n_items; qb += nwarps * (32 / GL)) {  // warp-uniform
    const int q = qb + lane / GL;
    int i = -1, vn = -1;
    long long tn = 0;
    bool ready = false;
    if (q < n_items) {
      i = listed ? clist[q] : q;
      if (gl < 3) vn = d.tri[3 * i + gl];  // the vertex this lane moves if i is ready, loaded early
      const long long ti = d.t[i];
      if (ti < Ts) {
        tn = ti + d.dt[i];
        ready = true;
        for (int base = d.sw_ptr[i], pe = d.sw_ptr[i + 1]; base < pe; base += GL * UN) {
          int jj[UN];
#pragma unroll
          for (int u = 0; u < UN; ++u) {
            const int p = base + u * GL + gl;
            jj[u] = p < pe ? d.sw[p] : -1;
          }
          bool bad = false;
#pragma unroll
          for (int u = 0; u < UN; ++u)
            if (jj[u] >= 0) {
              const long long tj = d.t[jj[u]];
              bad |= tj > tn || tn > tj + d.dt[jj[u]];
            }
          if (__any_sync(gmask, bad)) {
            ready = false;
            break;
          }
        }
      }
    }
    // ready list: one slot per ready candidate (its group's lane 0)
    const unsigned br = __ballot_sync(0xffffffffu, ready && gl == 0);
    int base_r = 0;
    if (lane == 0 && br) base_r = atomicAdd(&d.cnt->n_ready, __popc(br));
    base_r = __shfl_sync(0xffffffffu, base_r, 0);
    if (ready && gl == 0) {
      d.ready_list[base_r + __popc(br & lt)] = i;
      d.elem_ready[i] = epoch;
    }
    // its three vertices move to tn; the first to claim a node lists it
    bool claim = false;
    int n = -1;
    if (ready && gl < 3) {
      n = vn;
      d.ntn[n] = tn;
      claim = atomicExch(&d.node_moved[n], epoch) != epoch;
    }
    const unsigned bm = __ballot_sync(0xffffffffu, claim);
    int base_m = 0;
    if (lane == 0 && bm) base_m = atomicAdd(&d.cnt->n_moved, __popc(bm));
    base_m = __shfl_sync(0xffffffffu, base_m, 0);
    if (claim) d.moved_list[base_m + __popc(bm & lt)] = n;
  }
}

// End of a sweep: commit the moved nodes, list the next sweep's ready
// candidates (the total stencils of this sweep's ready elements), and in the
// last block to finish reset the per-sweep counters and advance the epoch.
__global__ void k_finish(Tab T, Dev d) {
  const int epoch = d.cnt->epoch;
  const int n_moved = d.cnt->n_moved;
  const int n_ready = d.cnt->n_ready;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  // loads before stores (a load after a store that may alias it waits for it)
  for (int q = gtid; q < n_moved; q += nth) {
    const int n = d.moved_list[q];
    const double x = d.nXn[2 * n], y = d.nXn[2 * n + 1];
    const long long tn = d.ntn[n];
    d.nX[2 * n] = x;
    d.nX[2 * n + 1] = y;
    d.nt[n] = tn;
  }
  if (!T.gts) {
    const int par = (epoch + 1) & 1;
    int* clist = d.cand_list + (size_t)par * d.ne;
    const int lane = threadIdx.x & 31;
    for (int q = gtid >> 5; q < n_ready; q += nth >> 5) {
      const int i = d.ready_list[q];
      for (int p = d.sw_ptr[i] + lane, pe = d.sw_ptr[i + 1]; p < pe; p += 96) {
        int jj[3];  // three chunks of the total stencil loaded before their atomics
#pragma unroll
        for (int u = 0; u < 3; ++u) jj[u] = p + 32 * u < pe ? d.sw[p + 32 * u] : -1;
#pragma unroll
        for (int u = 0; u < 3; ++u)
          if (jj[u] >= 0 && atomicExch(&d.cand_stamp[jj[u]], epoch) != epoch) {
            const int s2 = atomicAdd(&d.cnt->n_cand[par], 1);
            clist[s2] = jj[u];
          }
      }
    }
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&d.cnt->finish_blocks, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    Counters* c = d.cnt;
    if (!T.gts) c->cand_valid = 1;
    if (n_ready > 0) c->productive += 1;
    c->last_ready = n_ready;
    c->n_cand[epoch & 1] = 0;  // consumed by this sweep; refilled by the next one's finish
    c->n_ready = 0;
    c->n_moved = 0;
    c->surfaces += c->n_active;
    c->n_active = 0;
    c->n_touched = 0;
    c->sweeps += 1;
    c->finish_blocks = 0;
    c->epoch = epoch + 1;
  }
}

// Node solver with 8 lanes per moved node, one Voronoi element per lane
// (strided), partial sums combined by a fixed xor-shuffle tree.
template <int M>
__global__ void k_nodes_grp(Tab T, Dev d) {
  constexpr int Nt = M + 1, GS = 8;
  const int n_items = d.cnt->n_moved * GS;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_items; base += stride) {
    const int item = base + threadIdx.x;
    const int q = item / GS, lane = item % GS;
    double num0 = 0.0, num1 = 0.0, den = 0.0;
    int n = -1, ty = 0;
    double nnx = 0.0, nny = 0.0, x0 = 0.0, y0 = 0.0;
    if (item < n_items) {
      n = d.moved_list[q];
      const long long tk0 = d.nt[n], tk1 = d.ntn[n];
      if (lane == 0) {  // the node's own data, loaded beside the Voronoi loop's
        ty = d.node_type[n];
        nnx = d.node_n[2 * n];
        nny = d.node_n[2 * n + 1];
        x0 = d.nX[2 * n];
        y0 = d.nX[2 * n + 1];
      }
      for (int p = d.v2e_ptr[n] + lane, pe = d.v2e_ptr[n + 1]; p < pe; p += GS) {
        const int j = d.v2e[p];
        const int k = d.v2e_loc[p];
        const double mu = d.Q[4 * (size_t)j] * area6(d.X + 6 * (size_t)j);
        double D0 = 0.0, D1 = 0.0;
        const long long dtj = d.dt[j];
        if (dtj > 0) {
          const long long tj = d.t[j];
          const double idtj = 1.0 / (double)dtj;
          const double tau0 = (double)(tk0 - tj) * idtj;
          const double tau1 = (double)(tk1 - tj) * idtj;
          const double* vd = d.vdisp + ((size_t)j * 3 + k) * 2 * Nt;
          double a0 = vd[Nt - 1], a1 = vd[Nt - 1], b0 = vd[2 * Nt - 1], b1 = vd[2 * Nt - 1];
#pragma unroll
          for (int pp = Nt - 2; pp >= 0; --pp) {
            a0 = a0 * tau0 + vd[pp];
            a1 = a1 * tau1 + vd[pp];
            b0 = b0 * tau0 + vd[Nt + pp];
            b1 = b1 * tau1 + vd[Nt + pp];
          }
          const double dts = (double)dtj * d.etick[j];
          D0 = dts * (a1 * tau1 - a0 * tau0);
          D1 = dts * (b1 * tau1 - b0 * tau0);
        }
        num0 += mu * D0;
        num1 += mu * D1;
        den += mu;
      }
    }
#pragma unroll
    for (int off = GS / 2; off > 0; off >>= 1) {
      num0 += __shfl_xor_sync(0xffffffffu, num0, off, GS);
      num1 += __shfl_xor_sync(0xffffffffu, num1, off, GS);
      den += __shfl_xor_sync(0xffffffffu, den, off, GS);
    }
    if (item < n_items && lane == 0) {
      const double iden = 1.0 / den;
      double D0 = num0 * iden, D1 = num1 * iden;
      if (ty == 1) {
        const double nx = nnx, ny = nny;
        const double dn = D0 * nx + D1 * ny;
        D0 -= dn * nx;
        D1 -= dn * ny;
      } else if (ty == 2) {
        D0 = D1 = 0.0;
      } else if (ty == 3) {  // moves with the wall
        const double span = (double)(d.ntn[n] - d.nt[n]) * d.etick[d.v2e[d.v2e_ptr[n]]];
        D0 = T.wall_u * span;
        D1 = T.wall_v * span;
      }
      d.nXn[2 * n] = x0 + D0;
      d.nXn[2 * n + 1] = y0 + D1;
    }
  }
}

// edges with a moved endpoint, found through the moved nodes' incident edges
__global__ void k_edges(Dev d) {
  // 8 lanes per moved node, one incident edge per lane (strided)
  const int epoch = d.cnt->epoch;
  const int n_items = d.cnt->n_moved * 8;
  for (int item = blockIdx.x * blockDim.x + threadIdx.x; item < n_items; item += gridDim.x * blockDim.x) {
    const int n = d.moved_list[item >> 3];
    for (int p = d.n2e_ptr[n] + (item & 7), pe = d.n2e_ptr[n + 1]; p < pe; p += 8) {
      const int ed = d.n2e[p];
      const int ee[2] = {d.edge_elem[2 * ed], d.edge_elem[2 * ed + 1]};  // loaded beside the claim
      if (atomicExch(&d.edge_act[ed], epoch) == epoch) continue;
      const int slot = atomicAdd(&d.cnt->n_active, 1);
      d.active_list[slot] = ed;
      for (int k = 0; k < 2; ++k) {
        const int e = ee[k];
        if (e >= 0 && atomicExch(&d.elem_touch[e], epoch) != epoch) {
          const int s2 = atomicAdd(&d.cnt->n_touched, 1);
          d.touch_list[s2] = e;
        }
      }
    }
  }
}

// Exact state of the Kidder compression (Sec. 3.4, eqs. KidderIC, KidderEx)
// at (x, y, t): a particle starting at radius r sits at h(t) r with
// h = sqrt(1 - t^2/tau^2); density rho0(r)/h^2 with rho0^(gamma-1) linear in
// r^2 between the two frontiers, radial velocity h' r, pressure s0 rho^gamma;
// tau = sqrt((gamma-1)/2 (r_e0^2 - r_i0^2)/(c_e0^2 - c_i0^2)).
__device__ void kidder_state(const Tab& T, double x, double y, double t, double* q) {
  const double g = T.gamma, ri = T.kidder[0], re = T.kidder[1], s0 = T.kidder[4];
  const double ai = pow(T.kidder[2], g - 1.0), ae = pow(T.kidder[3], g - 1.0);
  const double ci2 = g * s0 * ai, ce2 = g * s0 * ae;
  const double tau2 = 0.5 * (g - 1.0) * (re * re - ri * ri) / (ce2 - ci2);
  const double h = sqrt(1.0 - t * t / tau2), dh = -t / (tau2 * h);
  const double R = sqrt(x * x + y * y), r = R / h;
  const double w = (r * r - ri * ri) / (re * re - ri * ri);
  const double rho = pow((1.0 - w) * ai + w * ae, 1.0 / (g - 1.0)) / (h * h);
  const double u = dh / h * x, v = dh / h * y;
  const double p = s0 * pow(rho, g);
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = p / (g - 1.0) + 0.5 * rho * (u * u + v * v);
}

// Rusanov-type ALE flux through the area-weighted space-time normal n
// (eq. rusanov): the largest |eigenvalue| of A_n^V times |n_xy| is
// |v.n_xy + n_t| + c |n_xy|.
__device__ __forceinline__ void rusanov(const Tab& T, const double* qm, const double* qp, const double* n,
                                        double* F) {
  // both sides' 1 / rho from one reciprocal
  const double rr = 1.0 / (qm[0] * qp[0]);
  double rim = qp[0] * rr, rip = qm[0] * rr;
  double um = qm[1] * rim, vm = qm[2] * rim, up = qp[1] * rip, vp = qp[2] * rip;
  double pm = (T.gamma - 1.0) * (qm[3] - 0.5 * (qm[1] * um + qm[2] * vm));
  double pp = (T.gamma - 1.0) * (qp[3] - 0.5 * (qp[1] * up + qp[2] * vp));
  // c |n_xy| as one square root per side
  double nn2 = n[0] * n[0] + n[1] * n[1];
  double cmn = sqrt(T.gamma * pm * rim * nn2), cpn = sqrt(T.gamma * pp * rip * nn2);
  double wm = um * n[0] + vm * n[1] + n[2], wp = up * n[0] + vp * n[1] + n[2];
  double sm = fabs(wm) + cmn, sp = fabs(wp) + cpn;
  double smax = fmax(sm, sp);
  // F~.n = f n_x + g n_y + q n_t = q (v.n_xy + n_t) + p (0, n_x, n_y, v.n_xy)
  double vnm = um * n[0] + vm * n[1], vnp = up * n[0] + vp * n[1];
  double Fm[4] = {qm[0] * wm, qm[1] * wm + pm * n[0], qm[2] * wm + pm * n[1], qm[3] * wm + pm * vnm};
  double Fp[4] = {qp[0] * wp, qp[1] * wp + pp * n[0], qp[2] * wp + pp * n[1], qp[3] * wp + pp * vnp};
#pragma unroll
  for (int v = 0; v < 4; ++v) F[v] = 0.5 * (Fm[v] + Fp[v]) - 0.5 * smax * (qp[v] - qm[v]);
}

// Osher-type ALE flux (eq. osher) on the straight path Psi(s) = q- + s (q+ -
// q-) (eq. path), the path integral by 3-point Gauss-Legendre quadrature:
// at each path node |A| dq = R |Lambda| L dq with the eigenvalues
// |n_xy| (u_n - c, u_n, u_n, u_n + c) + n_t of the ALE Jacobian and the
// eigenvectors R, L = R^-1 of dF/dQ.n, n = n_xy / |n_xy|.
__device__ __forceinline__ void osher(const Tab& T, const double* qm, const double* qp, const double* n,
                                      double* F) {
  const double g = T.gamma, gm1 = g - 1.0;
  double rim = 1.0 / qm[0], rip = 1.0 / qp[0];
  double um = qm[1] * rim, vm = qm[2] * rim, up = qp[1] * rip, vp = qp[2] * rip;
  double pm = gm1 * (qm[3] - 0.5 * (qm[1] * um + qm[2] * vm));
  double pp = gm1 * (qp[3] - 0.5 * (qp[1] * up + qp[2] * vp));
  double wm = um * n[0] + vm * n[1] + n[2], wp = up * n[0] + vp * n[1] + n[2];
  double vnm = um * n[0] + vm * n[1], vnp = up * n[0] + vp * n[1];
  const double nxy = sqrt(n[0] * n[0] + n[1] * n[1]);
  double nx = 1.0, ny = 0.0;
  if (nxy > 0.0) {
    const double inx = 1.0 / nxy;
    nx = n[0] * inx;
    ny = n[1] * inx;
  }
  double dq[4], D[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int v = 0; v < 4; ++v) dq[v] = qp[v] - qm[v];
  const double r15 = 0.38729833462074168852;  // sqrt(15) / 10
#pragma unroll
  for (int gq = 0; gq < 3; ++gq) {
    const double s = gq == 0 ? 0.5 - r15 : (gq == 1 ? 0.5 : 0.5 + r15);
    const double ws = gq == 1 ? 8.0 / 18.0 : 5.0 / 18.0;
    double q[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) q[v] = qm[v] + s * dq[v];
    const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
    const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
    const double a = sqrt(g * p * ir), ia = 1.0 / a, H = (q[3] + p) * ir;
    const double un = u * nx + v * ny, ut = -u * ny + v * nx, q2 = 0.5 * (u * u + v * v);
    const double b1 = gm1 * ia * ia, b2 = b1 * q2;
    // characteristic amplitudes L dq, scaled by |lambda|
    double c0 = 0.5 * (b2 + un * ia) * dq[0] - 0.5 * (b1 * u + nx * ia) * dq[1] - 0.5 * (b1 * v + ny * ia) * dq[2] +
                0.5 * b1 * dq[3];
    double c1 = (1.0 - b2) * dq[0] + b1 * u * dq[1] + b1 * v * dq[2] - b1 * dq[3];
    double c2 = -ut * dq[0] - ny * dq[1] + nx * dq[2];
    double c3 = 0.5 * (b2 - un * ia) * dq[0] - 0.5 * (b1 * u - nx * ia) * dq[1] - 0.5 * (b1 * v - ny * ia) * dq[2] +
                0.5 * b1 * dq[3];
    c0 *= ws * fabs(nxy * (un - a) + n[2]);
    c1 *= ws * fabs(nxy * un + n[2]);
    c2 *= ws * fabs(nxy * un + n[2]);
    c3 *= ws * fabs(nxy * (un + a) + n[2]);
    D[0] += c0 + c1 + c3;
    D[1] += (u - a * nx) * c0 + u * c1 - ny * c2 + (u + a * nx) * c3;
    D[2] += (v - a * ny) * c0 + v * c1 + nx * c2 + (v + a * ny) * c3;
    D[3] += (H - a * un) * c0 + q2 * c1 + ut * c2 + (H + a * un) * c3;
  }
  const double Fm[4] = {qm[0] * wm, qm[1] * wm + pm * n[0], qm[2] * wm + pm * n[1], qm[3] * wm + pm * vnm};
  const double Fp[4] = {qp[0] * wp, qp[1] * wp + pp * n[0], qp[2] * wp + pp * n[1], qp[3] * wp + pp * vnp};
#pragma unroll
  for (int v = 0; v < 4; ++v) F[v] = 0.5 * (Fm[v] + Fp[v]) - 0.5 * D[v];
}

// Per-edge data of a swept surface, formed once per edge (not once per Gauss
// point): its four corners (x, y, t in seconds: a, b at the old node times,
// b', a' at the new ones), the corner ticks, and for each side its element,
// local edge, time (ticks) and reciprocal step (0 for a zero step).
struct EdgeSetup {
  double P[4][3];
  double tk[4];
  double tL, itL, tR, itR, etL;
  int L, R, le, lr, bc;
};

// One lane per Gauss point: (M+1)^2 consecutive lanes per swept edge,
// 32 / (M+1)^2 edges per warp, the point contributions summed by a fixed
// shuffle tree within each edge's lanes.
template <int M>
__global__ void __launch_bounds__(kBlock) k_flux_grp(Tab T, Dev d) {
  // one thread per Gauss point, the block's EPB edges packed back to back
  // (an edge's points may span two warps: every lane of a warp FP64
  // instruction costs the pipe the same, used or not), the point sums
  // through shared memory in point order.  The per-edge set-up runs first,
  // one thread per edge, so that its FP64 work (tick conversions, the
  // sides' reciprocal steps) is issued once per edge instead of once per
  // Gauss point.
  constexpr int Nt = M + 1, NP = Nt * Nt, EPB = kBlock / NP;
  __shared__ double sGN[kBlock][7];
  __shared__ EdgeSetup sE[EPB];
  const int epoch = d.cnt->epoch;
  const int n_active = d.cnt->n_active;
  const int slot = threadIdx.x / NP, pt = threadIdx.x % NP;
  for (int first = blockIdx.x * EPB; first < n_active; first += gridDim.x * EPB) {
    for (int k = threadIdx.x; k < EPB; k += kBlock) {
      if (first + k >= n_active) continue;
      const int ed = d.active_list[first + k];
      const int a = d.edge_nodes[2 * ed], b = d.edge_nodes[2 * ed + 1];
      const int L = d.edge_elem[2 * ed], R = d.edge_elem[2 * ed + 1];
      const int le = d.edge_loc[2 * ed], lr = d.edge_loc[2 * ed + 1];
      const bool ma = d.node_moved[a] == epoch, mb = d.node_moved[b] == epoch;
      const int le1 = le == 2 ? 0 : le + 1;
      const double sax = d.cshift[6 * L + 2 * le], say = d.cshift[6 * L + 2 * le + 1];
      const double sbx = d.cshift[6 * L + 2 * le1], sby = d.cshift[6 * L + 2 * le1 + 1];
      const long long tL = d.t[L], dtL = d.dt[L];
      const double etL = d.etick[L];
      long long tR = 0, dtR = 0;
      if (R >= 0) {
        tR = d.t[R];
        dtR = d.dt[R];
      }
      EdgeSetup& E = sE[k];
      long long tk[4];
      E.P[0][0] = d.nX[2 * a] + sax; E.P[0][1] = d.nX[2 * a + 1] + say; tk[0] = d.nt[a];
      E.P[1][0] = d.nX[2 * b] + sbx; E.P[1][1] = d.nX[2 * b + 1] + sby; tk[1] = d.nt[b];
      if (mb) { E.P[2][0] = d.nXn[2 * b] + sbx; E.P[2][1] = d.nXn[2 * b + 1] + sby; tk[2] = d.ntn[b]; }
      else { E.P[2][0] = E.P[1][0]; E.P[2][1] = E.P[1][1]; tk[2] = tk[1]; }
      if (ma) { E.P[3][0] = d.nXn[2 * a] + sax; E.P[3][1] = d.nXn[2 * a + 1] + say; tk[3] = d.ntn[a]; }
      else { E.P[3][0] = E.P[0][0]; E.P[3][1] = E.P[0][1]; tk[3] = tk[0]; }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        E.tk[c] = (double)tk[c];
        E.P[c][2] = E.tk[c] * etL;
      }
      // a reciprocal costs the FP64 pipe half a divide
      E.tL = (double)tL;
      E.itL = dtL > 0 ? 1.0 / (double)dtL : 0.0;
      E.tR = (double)tR;
      E.itR = dtR > 0 ? 1.0 / (double)dtR : 0.0;
      E.etL = etL;
      E.L = L; E.R = R; E.le = le; E.lr = lr;
      E.bc = d.edge_bc[ed];
    }
    __syncthreads();
    const int q = first + slot;
    const bool valid = slot < EPB && q < n_active;
    double G[4] = {0, 0, 0, 0}, Nn[3] = {0, 0, 0};
    if (valid) {
      const EdgeSetup& E = sE[slot];
      const int gx = pt / Nt, gt = pt % Nt;
      const int L = E.L, R = E.R, le = E.le, lr = E.lr;
      double P[4][3];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) P[k][c] = E.P[k][c];
      const double chi = T.glx[gx], tau = T.glx[gt], wq = T.glw[gx] * T.glw[gt];
      double dchi[3], dtau[3], n[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dchi[c] = (1.0 - tau) * (P[1][c] - P[0][c]) + tau * (P[2][c] - P[3][c]);
        dtau[c] = (1.0 - chi) * (P[3][c] - P[0][c]) + chi * (P[2][c] - P[1][c]);
      }
      n[0] = dchi[1] * dtau[2] - dchi[2] * dtau[1];
      n[1] = dchi[2] * dtau[0] - dchi[0] * dtau[2];
      n[2] = dchi[0] * dtau[1] - dchi[1] * dtau[0];
      const double tt = (1 - chi) * (1 - tau) * E.tk[0] + chi * (1 - tau) * E.tk[1] + chi * tau * E.tk[2] +
                        (1 - chi) * tau * E.tk[3];
      double qm[4], qp[4];
      {
        const double tl = (tt - E.tL) * E.itL;
        const double* c0 = d.trace + ((((size_t)L * 3 + le) * Nt + gx) * Nt) * 4;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = c0[(Nt - 1) * 4 + v];
#pragma unroll
          for (int p = Nt - 2; p >= 0; --p) acc = acc * tl + c0[p * 4 + v];
          qm[v] = acc;
        }
      }
      const int bc = E.bc;
      if (R >= 0) {
        const double tr = (tt - E.tR) * E.itR;
        const double* c0 = d.trace + ((((size_t)R * 3 + lr) * Nt + (Nt - 1 - gx)) * Nt) * 4;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = c0[(Nt - 1) * 4 + v];
#pragma unroll
          for (int p = Nt - 2; p >= 0; --p) acc = acc * tr + c0[p * 4 + v];
          qp[v] = acc;
        }
      } else if (bc == 1) {
        // transmissive: the boundary element's sweep-start average (phase A
        // updates Q after this kernel), not the inner trace value, with
        // which a gas at rest beside the boundary grows from roundoff
#pragma unroll
        for (int v = 0; v < 4; ++v) qp[v] = d.Q[4 * (size_t)L + v];
      } else if (bc == 3) {
        // the exact Kidder state at the quadrature point
        const double px = (1 - chi) * (1 - tau) * P[0][0] + chi * (1 - tau) * P[1][0] + chi * tau * P[2][0] +
                          (1 - chi) * tau * P[3][0];
        const double py = (1 - chi) * (1 - tau) * P[0][1] + chi * (1 - tau) * P[1][1] + chi * tau * P[2][1] +
                          (1 - chi) * tau * P[3][1];
        kidder_state(T, px, py, tt * E.etL, qp);
      } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) qp[v] = qm[v];
        if (bc == 0 || bc == 2) {  // mirror the normal momentum relative to the wall
          const double wu = bc == 2 ? T.wall_u : 0.0, wv = bc == 2 ? T.wall_v : 0.0;
          const double nn = n[0] * n[0] + n[1] * n[1];
          if (nn > 0.0) {
            const double mn = ((qm[1] - qm[0] * wu) * n[0] + (qm[2] - qm[0] * wv) * n[1]) / nn;
            qp[1] = qm[1] - 2.0 * mn * n[0];
            qp[2] = qm[2] - 2.0 * mn * n[1];
            // same internal energy: a moving wall's mirror changes the kinetic energy
            if (bc == 2)
              qp[3] = qm[3] + 0.5 * (qp[1] * qp[1] + qp[2] * qp[2] - qm[1] * qm[1] - qm[2] * qm[2]) / qm[0];
          }
        }
      }
      double F[4];
      if (T.flux == 1) osher(T, qm, qp, n, F);
      else rusanov(T, qm, qp, n, F);
#pragma unroll
      for (int v = 0; v < 4; ++v) G[v] = wq * F[v];
#pragma unroll
      for (int c = 0; c < 3; ++c) Nn[c] = wq * n[c];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) sGN[threadIdx.x][v] = G[v];
#pragma unroll
    for (int c = 0; c < 3; ++c) sGN[threadIdx.x][4 + c] = Nn[c];
    __syncthreads();
    // one thread per (edge, component): the flux G (4) and the GCL vector (3)
    for (int it = threadIdx.x; it < EPB * 7; it += kBlock) {
      const int le = it / 7, k = it % 7, qq = first + le;
      if (qq >= n_active) continue;
      double acc = sGN[le * NP][k];
#pragma unroll
      for (int p2 = 1; p2 < NP; ++p2) acc += sGN[le * NP + p2][k];
      const int e2 = d.active_list[qq];
      if (k < 4) d.G[4 * (size_t)e2 + k] = acc;
      else d.N[4 * (size_t)e2 + k - 4] = acc;
    }
    __syncthreads();
  }
}

__global__ void k_update(Tab T, Dev d) {
  // Every load of a thread is issued before its first store: a load after a
  // store to memory that might alias it waits for the store, and this kernel
  // is a chain of dependent gathers whose round trips set its duration.
  const int epoch = d.cnt->epoch;
  const long long Ts = d.cnt->t_sync;
  const int n_touched = d.cnt->n_touched;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_touched; base += stride) {
    int q = base + threadIdx.x;
    bool upd = false;
    double gcl = 0.0;  // GCL residual of this thread's update (non-negative)
    if (q < n_touched) {
      const int i = d.touch_list[q];
      const bool ready = d.elem_ready[i] == epoch;
      int eds[3];
      bool act[3];
      double sg[3], Ge[3][4], Ne[3][3];
#pragma unroll
      for (int e = 0; e < 3; ++e) eds[e] = d.elem_edge[3 * i + e];
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        act[e] = d.edge_act[eds[e]] == epoch;
        sg[e] = d.edge_elem[2 * eds[e]] == i ? 1.0 : -1.0;
      }
#pragma unroll
      for (int e = 0; e < 3; ++e) {
#pragma unroll
        for (int v = 0; v < 4; ++v) Ge[e][v] = act[e] ? d.G[4 * (size_t)eds[e] + v] : 0.0;
#pragma unroll
        for (int c = 0; c < 3; ++c) Ne[e][c] = act[e] ? d.N[4 * (size_t)eds[e] + c] : 0.0;
      }
      double Qo[4], QMo[4], HMo[3];
#pragma unroll
      for (int v = 0; v < 4; ++v) { Qo[v] = d.Q[4 * i + v]; QMo[v] = d.QM[4 * i + v]; }
#pragma unroll
      for (int c = 0; c < 3; ++c) HMo[c] = d.HM[4 * i + c];
      if (ready) {
        upd = true;
        double Xo[6], Xn[6];
        int nd[3];
#pragma unroll
        for (int k = 0; k < 6; ++k) Xo[k] = d.X[6 * i + k];
#pragma unroll
        for (int k = 0; k < 3; ++k) nd[k] = d.tri[3 * i + k];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          Xn[2 * k] = d.nXn[2 * nd[k]] + d.cshift[6 * i + 2 * k];
          Xn[2 * k + 1] = d.nXn[2 * nd[k] + 1] + d.cshift[6 * i + 2 * k + 1];
        }
        const long long ti = d.t[i], dti = d.dt[i], ci = d.count[i];
        double Aold = area6(Xo), Anew = area6(Xn);
        double Qn[4];
        for (int v = 0; v < 4; ++v) {
          double acc = Aold * Qo[v];
          for (int e = 0; e < 3; ++e)
            if (act[e]) acc -= sg[e] * Ge[e][v];
          acc += QMo[v];
          Qn[v] = acc / Anew;
        }
        double res[3];
        for (int c = 0; c < 3; ++c) {
          double acc = 0.0;
          for (int e = 0; e < 3; ++e)
            if (act[e]) acc += sg[e] * Ne[e][c];
          res[c] = acc - HMo[c];
        }
        res[2] += Anew - Aold;
        gcl = fmax(fabs(res[0]), fmax(fabs(res[1]), fabs(res[2]))) / Aold;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          d.Q[4 * i + v] = Qn[v];
          d.QM[4 * i + v] = 0.0;
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) d.HM[4 * i + c] = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) d.X[6 * i + k] = Xn[k];
        d.t[i] = ti + dti;
        if (ti + dti >= Ts) atomicSub(&d.cnt->n_unfinished, 1);
        d.count[i] = ci + 1;
        if (!(Qn[0] > 0.0) || !(pressure(T, Qn) > 0.0) || !(Anew > 0.0)) set_error(d.cnt, -3, i);
      } else {
        double QMn[4], HMn[3];
        for (int v = 0; v < 4; ++v) {
          double acc = QMo[v];
          for (int e = 0; e < 3; ++e)
            if (act[e]) acc -= sg[e] * Ge[e][v];
          QMn[v] = acc;
        }
        for (int c = 0; c < 3; ++c) {
          double acc = HMo[c];
          for (int e = 0; e < 3; ++e)
            if (act[e]) acc -= sg[e] * Ne[e][c];
          HMn[c] = acc;
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) d.QM[4 * i + v] = QMn[v];
#pragma unroll
        for (int c = 0; c < 3; ++c) d.HM[4 * i + c] = HMn[c];
      }
    }
    unsigned um = __ballot_sync(0xffffffffu, upd);
    // the warp's largest residual (non-negative doubles order like their
    // bit patterns), one atomic per warp
    unsigned long long gb = (unsigned long long)__double_as_longlong(gcl);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, gb, off);
      gb = o > gb ? o : gb;
    }
    if ((threadIdx.x & 31) == 0 && um) atomicMax(&d.cnt->gcl_bits, gb);
    if ((threadIdx.x & 31) == 0 && um) {
      atomicAdd((unsigned long long*)&d.cnt->updates, (unsigned long long)__popc(um));
      atomicAdd((unsigned long long*)&d.cnt->updates_since_sync, (unsigned long long)__popc(um));
    }
  }
}

// ---------------------------------------------------------------------------
// virtual data of element j at time ti (ticks): eqs. virtGeom, virtCellaverage
template <int M>
__device__ __forceinline__ void virtual_data(const Tab& T, const Dev& d, int j, long long ti, double* Xv, double* Qv) {
  constexpr int Nt = M + 1;
  const long long tj = d.t[j], dtj = d.dt[j];
#pragma unroll
  for (int k = 0; k < 6; ++k) Xv[k] = d.X[6 * j + k];
  if (tj == ti || dtj == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) Qv[v] = d.Q[4 * j + v];
    return;
  }
  const double tau = (double)(ti - tj) * (1.0 / (double)dtj);  // a reciprocal costs half a divide
  const double dts = (double)dtj * d.etick[j];
  const double* vd = d.vdisp + (size_t)j * 6 * Nt;
#pragma unroll
  for (int kc = 0; kc < 6; ++kc) {
    const double* c0 = vd + kc * Nt;
    double acc = c0[Nt - 1];
#pragma unroll
    for (int p = Nt - 2; p >= 0; --p) acc = acc * tau + c0[p];
    Xv[kc] += dts * (acc * tau);
  }
  const double* av = d.avgc + (size_t)j * Nt * 4;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    double acc = av[(Nt - 1) * 4 + v];
#pragma unroll
    for (int p = Nt - 2; p >= 0; --p) acc = acc * tau + av[p * 4 + v];
    Qv[v] = acc;
  }
}

// predictor-derived tables of element i from qh[Nt][Mc][4]
template <int M>
__device__ __forceinline__ void write_products(const Tab& T, const Dev& d, int i, const double (*qh)[(M + 1) * (M + 2) / 2][4]) {
  constexpr int Mc = (M + 1) * (M + 2) / 2, Nt = M + 1;
  double* tr = d.trace + (size_t)i * 3 * Nt * Nt * 4;
  for (int e = 0; e < 3; ++e)
    for (int g = 0; g < Nt; ++g) {
      double val[Nt][4];
      for (int t = 0; t < Nt; ++t)
        for (int v = 0; v < 4; ++v) {
          double acc = 0.0;
          for (int s = 0; s < Mc; ++s) acc += T.Tr[e][g][s] * qh[t][s][v];
          val[t][v] = acc;
        }
      for (int p = 0; p < Nt; ++p)
        for (int v = 0; v < 4; ++v) {
          double acc = 0.0;
          for (int t = 0; t < Nt; ++t) acc += T.VtInv[p][t] * val[t][v];
          tr[((e * Nt + g) * Nt + p) * 4 + v] = acc;
        }
    }
  double* av = d.avgc + (size_t)i * Nt * 4;
  {
    double val[Nt][4];
    for (int t = 0; t < Nt; ++t)
      for (int v = 0; v < 4; ++v) {
        double acc = 0.0;
        for (int s = 0; s < Mc; ++s) acc += T.wavg[s] * qh[t][s][v];
        val[t][v] = acc;
      }
    for (int p = 0; p < Nt; ++p)
      for (int v = 0; v < 4; ++v) {
        double acc = 0.0;
        for (int t = 0; t < Nt; ++t) acc += T.VtInv[p][t] * val[t][v];
        av[p * 4 + v] = acc;
      }
  }
  double* vd = d.vdisp + (size_t)i * 6 * Nt;
  for (int k = 0; k < 3; ++k) {
    const int s = T.vnode[k];
    double vel[Nt][2];
    for (int t = 0; t < Nt; ++t) {
      double ir = 1.0 / qh[t][s][0];
      vel[t][0] = T.eulerian ? 0.0 : qh[t][s][1] * ir;
      vel[t][1] = T.eulerian ? 0.0 : qh[t][s][2] * ir;
    }
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p < Nt; ++p) {
        double acc = 0.0;
        for (int t = 0; t < Nt; ++t) acc += T.VtInv[p][t] * vel[t][c];
        vd[(k * 2 + c) * Nt + p] = acc / (p + 1);
      }
  }
}

template <int M>
__global__ void k_products(Tab T, Dev d) {
  constexpr int Mc = (M + 1) * (M + 2) / 2, Nt = M + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ne; i += gridDim.x * blockDim.x) {
    double q[Nt][Mc][4];
    const double* in = d.qhat + (size_t)i * Mc * Nt * 4;
    for (int t = 0; t < Nt; ++t)
      for (int s = 0; s < Mc; ++s)
        for (int v = 0; v < 4; ++v) q[t][s][v] = in[(t * Mc + s) * 4 + v];
    write_products<M>(T, d, i, q);
  }
}

// ---------------------------------------------------------------------------
// Cooperative predictor: one thread per (element, space-time node), G
// elements per 128-thread block, the element's nodal arrays in shared memory.
// ---------------------------------------------------------------------------
template <int M, int TH = 128>
struct PredShape {
  static constexpr int Mc = (M + 1) * (M + 2) / 2, Nt = M + 1, Nst = Mc * Nt;
  static constexpr int kThreads = TH;
  static constexpr int G = kThreads / Nst;
};

template <int M, int TH>
__global__ void __launch_bounds__(TH, TH >= 256 ? 2 : 3) k_predict_coop(Tab T, Dev d, int initial, int gts) {
  using S = PredShape<M, TH>;
  constexpr int Mc = S::Mc, Nt = S::Nt, Nst = S::Nst, G = S::G;
  __shared__ double sq[G][Nst][4], sf[G][Nst][4], sg[G][Nst][4], sP[G][Nst][4];
  __shared__ double sx[G][Nst][2], sV[G][Nst][2];
  // sTr: the 3 Nt rows of edge-trace weights (edge, Gauss point), then the
  // reference-average weights, so that traces and averages share one code path
  __shared__ double sDxi[Mc][Mc], sDeta[Mc][Mc], sB[Nt - 1][Nt], sDtau[Nt][Nt], sTr[3 * Nt + 1][Mc], sVt[Nt][Nt];
  __shared__ double sdts[G];
  __shared__ int sidx[G], sbad[G];
  for (int k = threadIdx.x; k < Mc * Mc; k += blockDim.x) {
    sDxi[k / Mc][k % Mc] = T.Dxi[k / Mc][k % Mc];
    sDeta[k / Mc][k % Mc] = T.Deta[k / Mc][k % Mc];
  }
  for (int k = threadIdx.x; k < (Nt - 1) * Nt; k += blockDim.x) sB[k / Nt][k % Nt] = T.B[k / Nt][k % Nt];
  for (int k = threadIdx.x; k < Nt * Nt; k += blockDim.x) {
    sDtau[k / Nt][k % Nt] = T.Dtau[k / Nt][k % Nt];
    sVt[k / Nt][k % Nt] = T.VtInv[k / Nt][k % Nt];
  }
  for (int k = threadIdx.x; k < 3 * Nt * Mc; k += blockDim.x) sTr[k / Mc][k % Mc] = T.Tr[k / (Nt * Mc)][(k / Mc) % Nt][k % Mc];
  for (int k = threadIdx.x; k < Mc; k += blockDim.x) sTr[3 * Nt][k] = T.wavg[k];
  const int n_ready = initial ? d.ne : d.cnt->n_ready;
  const long long gmin = d.cnt->gts_min;
  // thread -> (time slice t, element e, lattice node s).  A warp-wide FP64
  // instruction costs the FP64 pipe the same whatever number of its lanes is
  // active, so the tau = 0 nodes (full work in the first iteration only) and
  // the tau > 0 nodes (full work in the later ones) sit in separate warps:
  // the tau = 0 nodes of all G elements first, padded to a whole warp, when
  // that fits the block, otherwise after the tau > 0 nodes.
  constexpr int nBot = G * Mc, nTop = G * Mc * (Nt - 1), nBotPad = (nBot + 31) / 32 * 32;
  constexpr bool padBot = nBotPad + nTop <= TH;
  // When one element's tau > 0 nodes nearly fill a warp (30 of 32 lanes at
  // fourth order), each element gets a warp of its own: the warps of the
  // elements a round leaves empty (balanced rounds give a block fewer than G
  // elements) then issue no instruction at all.
  constexpr int nTopE = Mc * (Nt - 1);
  constexpr bool perWarp = nTopE > 16 && nTopE <= 32 && nBotPad + 32 * G <= TH;
  int t, rr;
  if (perWarp) {
    const int x = threadIdx.x;
    const int ew = (x - nBotPad) >> 5, k = (x - nBotPad) & 31;
    if (x < nBot) { t = 0; rr = x; }
    else if (x >= nBotPad && ew < G && k < nTopE) { t = 1 + k / Mc; rr = ew * Mc + k % Mc; }
    else { t = Nt; rr = 0; }
  } else if (padBot) {
    const int x = threadIdx.x;
    if (x < nBot) { t = 0; rr = x; }
    else if (x >= nBotPad && x < nBotPad + nTop) { t = 1 + (x - nBotPad) / nBot; rr = (x - nBotPad) % nBot; }
    else { t = Nt; rr = 0; }
  } else {
    const int x = threadIdx.x;
    if (x < nTop) { t = 1 + x / nBot; rr = x % nBot; }
    else if (x < nTop + nBot) { t = 0; rr = x - nTop; }
    else { t = Nt; rr = 0; }
  }
  const int e = t < Nt ? rr / Mc : G;
  const int s = rr % Mc, l = (t < Nt ? t : 0) * Mc + s;
  const double gm1 = T.gamma - 1.0;
  for (int consumed = 0; consumed < n_ready;) {
    // balanced rounds, as in the reconstruction
    const int per = min(G, (n_ready - consumed + (int)gridDim.x - 1) / (int)gridDim.x);
    const int base = consumed + (int)blockIdx.x * per;
    const int cnt = max(0, min(per, n_ready - base));
    consumed += per * (int)gridDim.x;
    if (cnt == 0) continue;  // block-uniform
    const int pos = base + e;
    const bool live = e < cnt;
    if (live && l == 0) {
      const int i = initial ? pos : d.ready_list[pos];
      long long dtk = d.dt[i];
      if ((gts || d.t[i] < T.Tsw) && dtk > 0) {
        dtk = gmin;
        d.dt[i] = dtk;
      }
      sidx[e] = i;
      sdts[e] = (double)dtk * d.etick[i];
      sbad[e] = 0;
    }
    __syncthreads();
    const int i = live ? sidx[e] : 0;
    const double dts = live ? sdts[e] : 0.0;
    const bool work = live && dts > 0.0;
    if (live) {
      const double* w0 = d.w0 + (size_t)pos * Mc * 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) sq[e][l][v] = w0[s * 4 + v];
      const double* X = d.X + 6 * (size_t)i;
      sx[e][l][0] = X[0] + (X[2] - X[0]) * T.lat[s][0] + (X[4] - X[0]) * T.lat[s][1];
      sx[e][l][1] = X[1] + (X[3] - X[1]) * T.lat[s][0] + (X[5] - X[1]) * T.lat[s][1];
    }
    __syncthreads();
    const double idt = work ? 1.0 / dts : 0.0;
    // tau = 0 node: its data and spatial metric never change, so after the
    // first iteration only the xi_t, eta_t terms of P are recomputed there
    double c_fs[4] = {0, 0, 0, 0}, c_Qx[4] = {0, 0, 0, 0}, c_Qe[4] = {0, 0, 0, 0};
    double c_xix = 0, c_xiy = 0, c_etx = 0, c_ety = 0;
    for (int it = 0; it < T.nit; ++it) {
      // Iteration 0 starts from w_h at every slice and a static geometry, so P
      // is the same on every slice: it is computed on the tau = 0 slice only.
      const bool full = work && (it == 0 ? t == 0 : t > 0);
      if (full) {  // nodal fluxes and mesh velocity at the own node
        const double* q = sq[e][l];
        const double ir = 1.0 / q[0], u = q[1] * ir, v = q[2] * ir;
        const double p = gm1 * (q[3] - 0.5 * (q[1] * u + q[2] * v));
        sf[e][l][0] = q[1]; sf[e][l][1] = q[1] * u + p; sf[e][l][2] = q[1] * v; sf[e][l][3] = u * (q[3] + p);
        sg[e][l][0] = q[2]; sg[e][l][1] = q[2] * u; sg[e][l][2] = q[2] * v + p; sg[e][l][3] = v * (q[3] + p);
        sV[e][l][0] = T.eulerian ? 0.0 : u;
        sV[e][l][1] = T.eulerian ? 0.0 : v;
      }
      __syncthreads();
      if (full && t > 0) {
        // tau > 0 node (later iterations): P at the own node (eq. pdef) with
        // the isoparametric metric (eq. Jac) first, then one contraction with
        // the combined weights D_xi xi_x + D_eta eta_x (and the y, t ones)
        double xx = 0, xe = 0, yx = 0, ye = 0;
#pragma unroll
        for (int r = 0; r < Mc; ++r) {
          const double a = sDxi[s][r], b = sDeta[s][r];
          const int lr = t * Mc + r;
          xx += a * sx[e][lr][0]; xe += b * sx[e][lr][0];
          yx += a * sx[e][lr][1]; ye += b * sx[e][lr][1];
        }
        double xt = 0.0, yt = 0.0;
#pragma unroll
        for (int u = 0; u < Nt; ++u) {
          xt += sDtau[t][u] * sx[e][u * Mc + s][0];
          yt += sDtau[t][u] * sx[e][u * Mc + s][1];
        }
        xt *= idt;
        yt *= idt;
        const double idet = 1.0 / (xx * ye - xe * yx);
        const double xix = ye * idet, xiy = -xe * idet, etx = -yx * idet, ety = xx * idet;
        const double xit = -(xix * xt + xiy * yt), ett = -(etx * xt + ety * yt);
        double Pv[4] = {0, 0, 0, 0};
#pragma unroll
        for (int r = 0; r < Mc; ++r) {
          const double a = sDxi[s][r], b = sDeta[s][r];
          const double wx = a * xix + b * etx, wy = a * xiy + b * ety, wt = a * xit + b * ett;
          const int lr = t * Mc + r;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            Pv[v] += wx * sf[e][lr][v];
            Pv[v] += wy * sg[e][lr][v];
            Pv[v] += wt * sq[e][lr][v];
          }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) sP[e][l][v] = -Pv[v];
      } else if (full) {  // tau = 0 node, first iteration: P (eq. pdef, eq. Jac) keeping its parts
        double Qx[4] = {0, 0, 0, 0}, Qe[4] = {0, 0, 0, 0}, fx[4] = {0, 0, 0, 0}, fe[4] = {0, 0, 0, 0};
        double gx[4] = {0, 0, 0, 0}, ge[4] = {0, 0, 0, 0};
        double xx = 0, xe = 0, yx = 0, ye = 0;
#pragma unroll
        for (int r = 0; r < Mc; ++r) {
          const double a = sDxi[s][r], b = sDeta[s][r];
          const int lr = t * Mc + r;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const double qv = sq[e][lr][v], fv = sf[e][lr][v], gv = sg[e][lr][v];
            Qx[v] += a * qv; Qe[v] += b * qv;
            fx[v] += a * fv; fe[v] += b * fv;
            gx[v] += a * gv; ge[v] += b * gv;
          }
          xx += a * sx[e][lr][0]; xe += b * sx[e][lr][0];
          yx += a * sx[e][lr][1]; ye += b * sx[e][lr][1];
        }
        double xt = 0.0, yt = 0.0;
        if (it > 0) {
#pragma unroll
          for (int u = 0; u < Nt; ++u) {
            xt += sDtau[t][u] * sx[e][u * Mc + s][0];
            yt += sDtau[t][u] * sx[e][u * Mc + s][1];
          }
          xt *= idt;
          yt *= idt;
        }
        const double idet = 1.0 / (xx * ye - xe * yx);
        const double xix = ye * idet, xiy = -xe * idet, etx = -yx * idet, ety = xx * idet;
        const double xit = -(xix * xt + xiy * yt), ett = -(etx * xt + ety * yt);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double fs = -(fx[v] * xix + fe[v] * etx + gx[v] * xiy + ge[v] * ety);
          sP[e][l][v] = fs - (Qx[v] * xit + Qe[v] * ett);
          if (t == 0) {
            c_fs[v] = fs;
            c_Qx[v] = Qx[v];
            c_Qe[v] = Qe[v];
          }
        }
        if (t == 0) {
          c_xix = xix; c_xiy = xiy; c_etx = etx; c_ety = ety;
        }
      } else if (work && t == 0) {  // tau = 0 node after the first iteration
        double xt = 0.0, yt = 0.0;
#pragma unroll
        for (int u = 0; u < Nt; ++u) {
          xt += sDtau[0][u] * sx[e][u * Mc + s][0];
          yt += sDtau[0][u] * sx[e][u * Mc + s][1];
        }
        xt *= idt;
        yt *= idt;
        const double xit = -(c_xix * xt + c_xiy * yt), ett = -(c_etx * xt + c_ety * yt);
#pragma unroll
        for (int v = 0; v < 4; ++v) sP[e][l][v] = c_fs[v] - (c_Qx[v] * xit + c_Qe[v] * ett);
      }
      __syncthreads();
      if (work && t > 0) {  // K_tau qhat = dt M P with the tau = 0 dofs known (eqs. CGfinal, newVertPos)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          double acc = 0.0;
#pragma unroll
          for (int u = 0; u < Nt; ++u) acc += sB[t - 1][u] * sP[e][(it == 0 ? 0 : u) * Mc + s][v];
          sq[e][l][v] = sq[e][s][v] + dts * acc;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          double acc = 0.0;
#pragma unroll
          for (int u = 0; u < Nt; ++u) acc += sB[t - 1][u] * sV[e][(it == 0 ? 0 : u) * Mc + s][c];
          sx[e][l][c] = sx[e][s][c] + dts * acc;
        }
      }
      __syncthreads();
    }
    // a non-positive density or pressure at any space-time node sends the
    // element back to w_h on every time slice
    if (work) {
      const double* q = sq[e][l];
      if (!(q[0] > 0.0) || !(gm1 * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]) > 0.0)) sbad[e] = 1;
    }
    __syncthreads();
    if (work && t > 0 && sbad[e]) {
#pragma unroll
      for (int v = 0; v < 4; ++v) sq[e][l][v] = sq[e][s][v];
    }
    __syncthreads();
    if (live) {
      double* out = d.qhat + ((size_t)i * Nst + l) * 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) out[v] = sq[e][l][v];
      // derived tables: edge traces and reference averages (one code path:
      // a weighted sum over each time slice's nodes, then the tau powers),
      // vertex displacements
      constexpr int nTr = 3 * Nt * 4, nItems = nTr + 4 + 6;
      for (int item = l; item < nItems; item += Nst) {
        if (item < nTr + 4) {
          const int row = item / 4, v = item % 4;  // row < 3 Nt: edge row / Nt, Gauss point row % Nt
          const double* wts = sTr[row];
          double val[Nt];
#pragma unroll
          for (int tt = 0; tt < Nt; ++tt) {
            double acc = 0.0;
#pragma unroll
            for (int r = 0; r < Mc; ++r) acc += wts[r] * sq[e][tt * Mc + r][v];
            val[tt] = acc;
          }
          double* dst = row < 3 * Nt ? d.trace + ((size_t)i * 3 * Nt + row) * Nt * 4 : d.avgc + (size_t)i * Nt * 4;
#pragma unroll
          for (int p = 0; p < Nt; ++p) {
            double acc = 0.0;
#pragma unroll
            for (int tt = 0; tt < Nt; ++tt) acc += sVt[p][tt] * val[tt];
            dst[p * 4 + v] = acc;
          }
        } else {
          const int kc = item - nTr - 4, k = kc / 2, c = kc % 2;
          const int sn = k == 0 ? 0 : (k == 1 ? M : Mc - 1);
          double vel[Nt];
#pragma unroll
          for (int tt = 0; tt < Nt; ++tt) {
            const double* q = sq[e][tt * Mc + sn];
            vel[tt] = T.eulerian ? 0.0 : q[1 + c] / q[0];
          }
          double* vd = d.vdisp + ((size_t)i * 6 + kc) * Nt;
#pragma unroll
          for (int p = 0; p < Nt; ++p) {
            double acc = 0.0;
#pragma unroll
            for (int tt = 0; tt < Nt; ++tt) acc += sVt[p][tt] * vel[tt];
            vd[p] = acc * (1.0 / (p + 1));  // p is unrolled: a constant factor
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Cooperative reconstruction: G ready elements per 256-thread block; each
// phase flattens its work items over the block (stencil members, normal-
// equation entries, stencils, characteristic fields, output nodes).
// ---------------------------------------------------------------------------
template <int M>
constexpr int recon_g_default() { return M == 1 ? 16 : (M == 2 ? 8 : 4); }

template <int M, int GG = recon_g_default<M>()>
struct ReconShape {
  static constexpr int Mc = (M + 1) * (M + 2) / 2, NU = Mc - 1, NE = 2 * Mc;
  static constexpr int MaxU = kNSten * (NE - 1);
  static constexpr int G = GG;
  // the default shape on 256 threads; half the elements on 128 threads (the
  // same threads per element, twice the blocks and barrier domains per SM)
  static constexpr int kThreads = GG < recon_g_default<M>() ? 128 : 256;
  static constexpr int NL = NU * (NU + 1) / 2;      // lower triangle of the normal matrix
  static constexpr int NN = NL + 4 * NU;           // + right-hand sides
  static constexpr int RW = NU + 4;                 // row: basis averages, then Q~ - Q_i
  static constexpr size_t oRow = 0;
  static constexpr size_t oNrm = oRow + (size_t)G * (MaxU + 1) * RW;
  static constexpr size_t oC = oNrm + (size_t)G * kNSten * NN;
  static constexpr size_t oCh = oC + (size_t)G * kNSten * NU * 4;
  static constexpr size_t oSig = oCh + (size_t)G * kNSten * NU * 4;
  static constexpr size_t oWc = oSig + (size_t)G * kNSten * 4;
  static constexpr size_t oCv = oWc + (size_t)G * NU * 4;
  static constexpr size_t oRL = oCv + (size_t)G * NU * 4;
  static constexpr size_t oEl = oRL + (size_t)G * 32;   // X(6), Q(4), Jinv(4)
  static constexpr size_t oDt = oEl + (size_t)G * 16;
  static constexpr size_t oBn = oDt + (size_t)G * 4;    // Bnod [Mc][NU]
  static constexpr size_t nDbl = oBn + (size_t)Mc * NU;
  static constexpr size_t nInt = 5 * G + 1 + G * kNSten;  // i, pos-valid, u0, nU, prefix[G+1], ok[G][7]
  static constexpr size_t bytes = nDbl * 8 + nInt * 4 + (size_t)G * kNSten * NE;
};

template <int M, int GG>
__global__ void __launch_bounds__(ReconShape<M, GG>::kThreads, 512 / ReconShape<M, GG>::kThreads)
k_recon_coop(Tab T, Dev d, int initial) {
  using S = ReconShape<M, GG>;
  constexpr int Mc = S::Mc, NU = S::NU, NE = S::NE, MaxU = S::MaxU, G = S::G, NL = S::NL, NN = S::NN, RW = S::RW;
  extern __shared__ double smem[];
  double* sRow = smem + S::oRow;
  double* sNrm = smem + S::oNrm;
  double* sC = smem + S::oC;
  double* sCh = smem + S::oCh;
  double* sSig = smem + S::oSig;
  double* sWc = smem + S::oWc;
  double* sCv = smem + S::oCv;
  double* sRL = smem + S::oRL;
  double* sEl = smem + S::oEl;
  double* sDt = smem + S::oDt;
  double* sBn = smem + S::oBn;
  int* sI = reinterpret_cast<int*>(smem + S::nDbl);
  int* sVal = sI + G;
  int* sU0 = sVal + G;
  int* sNU = sU0 + G;
  int* sPre = sNU + G;            // G + 1
  int* sOk = sPre + G + 1;        // G * 7
  unsigned char* sSt = reinterpret_cast<unsigned char*>(sOk + G * kNSten);
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int k = tid; k < Mc * NU; k += nth) sBn[k] = T.Bnod[k / NU][k % NU];
  const int n_ready = initial ? d.ne : d.cnt->n_ready;
  const long long Ts = d.cnt->t_sync;
  for (int consumed = 0; consumed < n_ready;) {
    // balanced rounds: every block takes the same number of elements (at
    // most G) per round, so that the elements of the last round spread over
    // all blocks instead of stacking on a few of them
    const int per = min(G, (n_ready - consumed + (int)gridDim.x - 1) / (int)gridDim.x);
    const int base = consumed + (int)blockIdx.x * per;
    const int cnt = max(0, min(per, n_ready - base));
    consumed += per * (int)gridDim.x;
    if (cnt == 0) continue;  // block-uniform
    // P0: element set-up
    if (tid < G) {
      const int e = tid, pos = base + e;
      const bool v = e < cnt;
      sVal[e] = v;
      int nU = 0;
      if (v) {
        const int i = initial ? pos : d.ready_list[pos];
        sI[e] = i;
        double* el = sEl + e * 16;
        for (int k = 0; k < 6; ++k) el[k] = d.X[6 * (size_t)i + k];
        for (int k = 0; k < 4; ++k) el[6 + k] = d.Q[4 * (size_t)i + k];
        const double ja = el[2] - el[0], jb = el[4] - el[0], jc = el[3] - el[1], jd = el[5] - el[1];
        const double idet = 1.0 / (ja * jd - jb * jc);
        el[10] = jd * idet; el[11] = -jb * idet; el[12] = -jc * idet; el[13] = ja * idet;
        sU0[e] = d.u_ptr[i];
        nU = d.u_ptr[i + 1] - sU0[e];
        for (int s = 0; s < kNSten; ++s) sOk[e * kNSten + s] = d.sten_ok[(size_t)i * kNSten + s];
      }
      sNU[e] = nU;
    }
    __syncthreads();
    if (tid == 0) {
      sPre[0] = 0;
      for (int e = 0; e < G; ++e) sPre[e + 1] = sPre[e] + (sVal[e] ? sNU[e] : 0);
    }
    for (int k = tid; k < G * kNSten * NE; k += nth) {
      const int e = k / (kNSten * NE);
      sSt[k] = sVal[e] ? d.sten[(size_t)sI[e] * kNSten * NE + k % (kNSten * NE)] : 0;
    }
    __syncthreads();
    // P1: rows of the least-squares systems (virtual data, eqs. virtGeom,
    // virtCellaverage, intConsRec), then the time-step candidates
    // (eq. timestep) on the last threads of the block, so that the warps
    // holding rows do not also run the time-step code with a few lanes
    for (int item = tid; item < sPre[G]; item += nth) {
      int e = 0;
      while (item >= sPre[e + 1]) ++e;
      const int u = item - sPre[e];
      const double* el = sEl + e * 16;
      const long long ti = d.t[sI[e]];
      double Xv[6], Qv[4];
      {
        const int q = sU0[e] + u;
        const int j = d.u_elem[q];
        virtual_data<M>(T, d, j, ti, Xv, Qv);
        const double sx = d.u_shift[2 * (size_t)q], sy = d.u_shift[2 * (size_t)q + 1];
        double xr[3], yr[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double px = Xv[2 * k] + sx - el[0], py = Xv[2 * k + 1] + sy - el[1];
          xr[k] = el[10] * px + el[11] * py - (1.0 / 3.0);
          yr[k] = el[12] * px + el[13] * py - (1.0 / 3.0);
        }
        // averages of the monomials over the virtual member (a straight
        // triangle) in closed form: with the centroid c and the vertex
        // offsets u_k = v_k - c, the second central moments are
        // (1/12) sum_k u_k u_k^T and the third (1/30) sum_k u_k (x) u_k (x) u_k,
        // so E[x^2] = c_x^2 + S_xx, E[x^2 y] = c_x^2 c_y + c_y S_xx + 2 c_x S_xy
        // + T_xxy, ...  (what the degree-M quadrature gives, with fewer
        // operations)
        double row[NU];
        const double cx = (xr[0] + xr[1] + xr[2]) * (1.0 / 3.0), cy = (yr[0] + yr[1] + yr[2]) * (1.0 / 3.0);
        row[0] = cx;
        row[1] = cy;
        if constexpr (M >= 2) {
          double ux[3], uy[3];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            ux[k] = xr[k] - cx;
            uy[k] = yr[k] - cy;
          }
          const double sxx = (ux[0] * ux[0] + ux[1] * ux[1] + ux[2] * ux[2]) * (1.0 / 12.0);
          const double sxy = (ux[0] * uy[0] + ux[1] * uy[1] + ux[2] * uy[2]) * (1.0 / 12.0);
          const double syy = (uy[0] * uy[0] + uy[1] * uy[1] + uy[2] * uy[2]) * (1.0 / 12.0);
          row[2] = cx * cx + sxx;
          row[3] = cx * cy + sxy;
          row[4] = cy * cy + syy;
          if constexpr (M >= 3) {
            double txxx = 0.0, txxy = 0.0, txyy = 0.0, tyyy = 0.0;
#pragma unroll
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
        double* dst = sRow + ((size_t)e * (MaxU + 1) + u + 1) * RW;
#pragma unroll
        for (int a = 0; a < NU; ++a) dst[a] = row[a] - T.mbar[a];
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[NU + v] = Qv[v] - el[6 + v];
      }
    }
    for (int item = nth - 1 - tid; item < G * 4; item += nth) {
      const int e = item / 4, k = item % 4;
      if (!sVal[e]) continue;
      const int i = sI[e];
      const long long ti = d.t[i];
      double Xv[6], Qv[4];
      {
        const int j = k == 0 ? i : d.nbr[3 * (size_t)i + k - 1];
        double dtc = DBL_MAX;
        if (j >= 0 && ti < Ts) {
          virtual_data<M>(T, d, j, ti, Xv, Qv);
          double per = 0.0;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) {
            const int k1 = kk == 2 ? 0 : kk + 1;
            const double dx = Xv[2 * k1] - Xv[2 * kk], dy = Xv[2 * k1 + 1] - Xv[2 * kk + 1];
            per += sqrt(dx * dx + dy * dy);
          }
          const double dd = 4.0 * area6(Xv) / per;
          const double uu = Qv[1] / Qv[0], vv = Qv[2] / Qv[0];
          double vel = sqrt(uu * uu + vv * vv);
          if (k == 0)  // an element on a moving wall counts the wall's speed
            for (int e2 = 0; e2 < 3; ++e2)
              if (d.edge_bc[d.elem_edge[3 * (size_t)i + e2]] == 2) vel = fmax(vel, T.wall_speed);
          const double lam = vel + sqrt(T.gamma * pressure(T, Qv) / Qv[0]);
          dtc = (ti < T.Tsw ? T.cfl_start : T.cfl) * dd / lam;
          if (!(dtc > 0.0)) dtc = -1.0;
        }
        sDt[e * 4 + k] = dtc;
      }
    }
    __syncthreads();
    // P2: normal equations of every stencil
    for (int item = tid; item < G * kNSten * NN; item += nth) {
      const int e = item / (kNSten * NN), s = (item / NN) % kNSten, q = item % NN;
      if (!sVal[e] || !sOk[e * kNSten + s]) continue;
      int a, b, v = -1;
      if (q < NL) {
        a = 0;
        while ((a + 1) * (a + 2) / 2 <= q) ++a;
        b = q - a * (a + 1) / 2;
      } else {
        a = (q - NL) / 4;
        v = (q - NL) % 4;
        b = NU + v;
      }
      const unsigned char* st = sSt + (e * kNSten + s) * NE;
      const double* R0 = sRow + (size_t)e * (MaxU + 1) * RW;
      double acc = 0.0;
#pragma unroll
      for (int m = 1; m < NE; ++m) {
        const double* r = R0 + (size_t)st[m] * RW;
        acc += r[a] * r[b];
      }
      sNrm[(e * kNSten + s) * NN + q] = acc;
    }
    __syncthreads();
    // P3a: Cholesky factorisation N = L L^T per stencil, in place; the
    // diagonal keeps 1 / L_aa
    for (int item = tid; item < G * kNSten; item += nth) {
      const int e = item / kNSten, s = item % kNSten;
      if (!sVal[e] || !sOk[e * kNSten + s]) continue;
      double* nm = sNrm + (size_t)item * NN;
      double L[NU][NU];
#pragma unroll
      for (int a = 0; a < NU; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) L[a][b] = nm[a * (a + 1) / 2 + b];
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        double dd = L[a][a];
#pragma unroll
        for (int k = 0; k < a; ++k) dd -= L[a][k] * L[a][k];
        const double il = rsqrt(dd);
        L[a][a] = il;
#pragma unroll
        for (int b = a + 1; b < NU; ++b) {
          double v = L[b][a];
#pragma unroll
          for (int k = 0; k < a; ++k) v -= L[b][k] * L[a][k];
          L[b][a] = v * il;
        }
      }
#pragma unroll
      for (int a = 0; a < NU; ++a)
#pragma unroll
        for (int b = 0; b <= a; ++b) nm[a * (a + 1) / 2 + b] = L[a][b];
    }
    __syncthreads();
    // P3b: the two triangular solves, one right-hand side per item, then one
    // step of the corrected semi-normal equations (Bjorck): r = b - A y over
    // the stencil's rows, solve L L^T dy = A^T r with the same factor,
    // y += dy.  The normal equations square the condition number of A; the
    // correction brings y to the accuracy of an orthogonal factorisation.
    for (int item = tid; item < G * kNSten * 4; item += nth) {
      const int es = item / 4, v = item % 4, e = es / kNSten, s = es % kNSten;
      if (!sVal[e] || !sOk[e * kNSten + s]) continue;
      const double* nm = sNrm + (size_t)es * NN;
      double* cs = sC + (size_t)es * NU * 4;
      const unsigned char* st = sSt + es * NE;
      const double* R0 = sRow + (size_t)e * (MaxU + 1) * RW;
      double y[NU], z[NU];
#pragma unroll
      for (int a = 0; a < NU; ++a) z[a] = nm[NL + a * 4 + v];
#pragma unroll
      for (int pass = 0; pass < 2; ++pass) {
#pragma unroll
        for (int a = 0; a < NU; ++a) {
          double acc = z[a];
#pragma unroll
          for (int k = 0; k < a; ++k) acc -= nm[a * (a + 1) / 2 + k] * z[k];
          z[a] = acc * nm[a * (a + 1) / 2 + a];
        }
#pragma unroll
        for (int a = NU - 1; a >= 0; --a) {
          double acc = z[a];
#pragma unroll
          for (int k = a + 1; k < NU; ++k) acc -= nm[k * (k + 1) / 2 + a] * z[k];
          z[a] = acc * nm[a * (a + 1) / 2 + a];
        }
        if (pass == 0) {
#pragma unroll
          for (int a = 0; a < NU; ++a) { y[a] = z[a]; z[a] = 0.0; }
#pragma unroll
          for (int m = 1; m < NE; ++m) {
            const double* r = R0 + (size_t)st[m] * RW;
            double res = r[NU + v];
#pragma unroll
            for (int a = 0; a < NU; ++a) res -= r[a] * y[a];
#pragma unroll
            for (int a = 0; a < NU; ++a) z[a] += r[a] * res;
          }
        } else {
#pragma unroll
          for (int a = 0; a < NU; ++a) y[a] += z[a];
        }
      }
#pragma unroll
      for (int a = 0; a < NU; ++a) cs[a * 4 + v] = y[a];
    }
    __syncthreads();
    // P4: characteristic fields of dF/dQ.n, n along the density gradient of
    // the central-stencil polynomial at the centroid (its linear coefficients)
    if (tid < G && sVal[tid]) {
      const int e = tid;
      const double* el = sEl + e * 16;
      const double* c0 = sC + (size_t)(e * kNSten) * NU * 4;
      const double gx = c0[0 * 4] * el[10] + c0[1 * 4] * el[12];
      const double gy = c0[0 * 4] * el[11] + c0[1 * 4] * el[13];
      // on G lanes of one warp: three reciprocals and two square roots, no
      // divides (each costs the warp's full FP64 issue)
      const double gn = sqrt(gx * gx + gy * gy);
      double nx = 1.0, ny = 0.0;
      if (gn > 0.0) {
        const double ign = 1.0 / gn;
        nx = gx * ign;
        ny = gy * ign;
      }
      const double g = T.gamma, rho = el[6], ir = 1.0 / rho, u = el[7] * ir, v = el[8] * ir;
      const double p = (g - 1.0) * (el[9] - 0.5 * rho * (u * u + v * v));
      const double a = sqrt(g * p * ir), H = (el[9] + p) * ir, un = u * nx + v * ny, ut = -u * ny + v * nx;
      const double ia = 1.0 / a, q2 = 0.5 * (u * u + v * v), b1 = (g - 1.0) * ia * ia, b2 = b1 * q2;
      double* R = sRL + e * 32;
      double* Lm = R + 16;
      R[0] = 1; R[1] = 1; R[2] = 0; R[3] = 1;
      R[4] = u - a * nx; R[5] = u; R[6] = -ny; R[7] = u + a * nx;
      R[8] = v - a * ny; R[9] = v; R[10] = nx; R[11] = v + a * ny;
      R[12] = H - a * un; R[13] = q2; R[14] = ut; R[15] = H + a * un;
      Lm[0] = 0.5 * (b2 + un * ia); Lm[1] = -0.5 * (b1 * u + nx * ia); Lm[2] = -0.5 * (b1 * v + ny * ia); Lm[3] = 0.5 * b1;
      Lm[4] = 1.0 - b2; Lm[5] = b1 * u; Lm[6] = b1 * v; Lm[7] = -b1;
      Lm[8] = -ut; Lm[9] = -ny; Lm[10] = nx; Lm[11] = 0.0;
      Lm[12] = 0.5 * (b2 - un * ia); Lm[13] = -0.5 * (b1 * u - nx * ia); Lm[14] = -0.5 * (b1 * v - ny * ia); Lm[15] = 0.5 * b1;
    }
    __syncthreads();
    // P5: characteristic coefficients and oscillation indicators (eq. weno)
    for (int item = tid; item < G * kNSten * 4; item += nth) {
      const int e = item / (kNSten * 4), s = (item / 4) % kNSten, r = item % 4;
      if (!sVal[e] || !sOk[e * kNSten + s]) continue;
      const double* Lr = sRL + e * 32 + 16 + r * 4;
      const double* cs = sC + (size_t)(e * kNSten + s) * NU * 4;
      double* ch = sCh + (size_t)(e * kNSten + s) * NU * 4;
      double cc[NU];
#pragma unroll
      for (int l = 0; l < NU; ++l) {
        cc[l] = Lr[0] * cs[l * 4] + Lr[1] * cs[l * 4 + 1] + Lr[2] * cs[l * 4 + 2] + Lr[3] * cs[l * 4 + 3];
        ch[l * 4 + r] = cc[l];
      }
      double sg = 0.0;
#pragma unroll
      for (int a = 0; a < NU; ++a) {
        double acc = 0.0;
#pragma unroll
        for (int b = a; b < NU; ++b) acc += T.SigU[a][b] * cc[b];
        sg += acc * acc;
      }
      sSig[(e * kNSten + s) * 4 + r] = sg;
    }
    __syncthreads();
    // P6: nonlinear weights (one item per element, stencil and field; the
    // weight overwrites its sigma), then the weighted characteristic
    // coefficients (one item per element, coefficient and field)
    for (int item = tid; item < G * kNSten * 4; item += nth) {
      const int e = item / (kNSten * 4), s = (item / 4) % kNSten;
      if (!sVal[e]) continue;
      double om = 0.0;
      if (sOk[e * kNSten + s]) {
        const double e1 = sSig[item] + 1e-14;
        const double e2 = e1 * e1, e4 = e2 * e2, e8 = e4 * e4;
        om = (s == 0 ? 1e5 : 1.0) / e8;
      }
      sSig[item] = om;
    }
    __syncthreads();
    for (int item = tid; item < G * NU * 4; item += nth) {
      const int e = item / (NU * 4), l = (item / 4) % NU, r = item % 4;
      if (!sVal[e]) continue;
      const double* om = sSig + (size_t)e * kNSten * 4 + r;
      double tot = 0.0;
#pragma unroll
      for (int s = 0; s < kNSten; ++s)
        if (sOk[e * kNSten + s]) tot += om[4 * s];
      const double itot = 1.0 / tot;
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < kNSten; ++s)
        if (sOk[e * kNSten + s]) acc += (om[4 * s] * itot) * sCh[((size_t)(e * kNSten + s) * NU + l) * 4 + r];
      sWc[(e * NU + l) * 4 + r] = acc;
    }
    __syncthreads();
    // P7: back to conserved variables
    for (int item = tid; item < G * NU * 4; item += nth) {
      const int e = item / (NU * 4), l = (item / 4) % NU, v = item % 4;
      if (!sVal[e]) continue;
      const double* Rv = sRL + e * 32 + v * 4;
      const double* wc = sWc + (e * NU + l) * 4;
      sCv[(e * NU + l) * 4 + v] = Rv[0] * wc[0] + Rv[1] * wc[1] + Rv[2] * wc[2] + Rv[3] * wc[3];
    }
    __syncthreads();
    // P8: nodal values of w_h for the predictor, and the new local time step
    double* sW0 = sCh;  // free after P6: [G][Mc][4]
    for (int item = tid; item < G * (Mc * 4 + 1); item += nth) {
      const int e = item / (Mc * 4 + 1), k = item % (Mc * 4 + 1);
      if (!sVal[e]) continue;
      const int i = sI[e];
      if (k < Mc * 4) {
        const int s = k / 4, v = k % 4;
        double acc = sEl[e * 16 + 6 + v];
#pragma unroll
        for (int l = 0; l < NU; ++l) acc += sBn[s * NU + l] * sCv[(e * NU + l) * 4 + v];
        sW0[(e * Mc + s) * 4 + v] = acc;
      } else {
        const long long ti = d.t[i];
        long long tks = 0;
        if (ti < Ts) {
          double best = DBL_MAX;
          bool bad = false;
          for (int c = 0; c < 4; ++c) {
            const double v = sDt[e * 4 + c];
            if (v < 0.0) bad = true;
            best = fmin(best, v);
          }
          if (bad || !(best > 0.0)) {
            set_error(d.cnt, -3, i);
            best = d.etick[i];
          }
          const double rt = floor(best / d.etick[i]);
          const bool start = ti < T.Tsw;  // global-step start-up
          const long long end = start ? (T.Tsw < Ts ? T.Tsw : Ts) : Ts;
          tks = rt > (double)(end - ti) ? end - ti : (long long)rt;
          if (tks < 1) tks = 1;
          if (T.gts || start) atomicMin(&d.cnt->gts_min, tks);
        }
        if (d.sched_mode) {  // frozen schedule: record or replay this update's step
          const long long ci = d.count[i];
          if (ci >= d.sched_k) {
            set_error(d.cnt, -7, i);
          } else {
            long long* slot = d.sched_log + (size_t)i * d.sched_k + ci;
            if (d.sched_mode == 1) *slot = tks;
            else tks = *slot;
          }
        }
        d.dt[i] = tks;
      }
    }
    __syncthreads();
    // P9: positivity scaling of w_h at the lattice nodes (density first, then
    // pressure through its chord bound; the scaling of Zhang and Shu), then
    // the nodal values go to the predictor.  Per pass: one candidate theta per
    // node, the element's minimum, the scaling.
    for (int pass = 0; pass < 2; ++pass) {
      double* cand = sSig;  // [G][Mc], free after P6
      for (int item = tid; item < G * Mc; item += nth) {
        const int e = item / Mc;
        if (!sVal[e]) continue;
        const double* Qi = sEl + e * 16 + 6;
        const double* ws = sW0 + (size_t)item * 4;
        double th = 1.0;
        if (pass == 0) {
          const double rho_min = 1e-8 * Qi[0];
          if (ws[0] < rho_min) th = (Qi[0] - rho_min) / (Qi[0] - ws[0]);
        } else {
          const double p_i = pressure(T, Qi), p_min = 1e-8 * p_i, ps = pressure(T, ws);
          if (ps < p_min) th = (p_i - p_min) / (p_i - ps);
        }
        cand[item] = th;
      }
      __syncthreads();
      for (int e = tid; e < G; e += nth) {
        double theta = 1.0;
        if (sVal[e])
          for (int k = 0; k < Mc; ++k) theta = fmin(theta, cand[e * Mc + k]);
        sDt[e * 4] = theta;  // free after P8
      }
      __syncthreads();
      for (int item = tid; item < G * Mc * 4; item += nth) {
        const int e = item / (Mc * 4);
        const double theta = sDt[e * 4];
        if (!sVal[e] || !(theta < 1.0)) continue;
        const double qi = sEl[e * 16 + 6 + item % 4];
        sW0[item] = qi + theta * (sW0[item] - qi);
      }
      __syncthreads();
    }
    for (int item = tid; item < G * Mc * 4; item += nth) {
      const int e = item / (Mc * 4);
      if (!sVal[e]) continue;
      d.w0[(size_t)(base + e) * Mc * 4 + item % (Mc * 4)] = sW0[item];
    }
    __syncthreads();
  }
}

// A new sync time Tn below the current one: every element whose step crosses
// Tn takes the step Tn - t instead and is listed (with its tau = 0 dofs, the
// scaled WENO values, as the predictor's nodal input) for a new predictor.
template <int M>
__global__ void k_sync_cut(Dev d, long long Tn) {
  constexpr int Mc = (M + 1) * (M + 2) / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ne; i += gridDim.x * blockDim.x) {
    const long long ti = d.t[i];
    if (!(ti < Tn && ti + d.dt[i] > Tn)) continue;
    d.dt[i] = Tn - ti;
    atomicMin(&d.cnt->gts_min, Tn - ti);
    const int slot = atomicAdd(&d.cnt->n_ready, 1);
    d.ready_list[slot] = i;
    const double* q0 = d.qhat + (size_t)i * (Mc * (M + 1)) * 4;
    double* w = d.w0 + (size_t)slot * Mc * 4;
#pragma unroll
    for (int k = 0; k < Mc * 4; ++k) w[k] = q0[k];
  }
}

// A new sync time above the current one Told: the elements stopped at Told
// are listed for their phase B.
__global__ void k_sync_resume(Dev d, long long Told) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ne; i += gridDim.x * blockDim.x)
    if (d.t[i] == Told) d.ready_list[atomicAdd(&d.cnt->n_ready, 1)] = i;
}

__global__ void k_sync_done(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    d.cnt->n_ready = 0;
    d.cnt->gts_min = LLONG_MAX;
    d.cnt->cand_valid = 0;  // new steps: the next sweep tests every element
  }
}

__global__ void k_fill_counters_initial(Dev d) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    d.cnt->gts_min = LLONG_MAX;
    d.cnt->err_code = 0;
  }
}

// The reconstruction and predictor grids cover every element (the pre-
// processing phase) or bpsm blocks per SM that loop over the ready list.
template <int M, int GG>
void launch_recon_g(const Tab& T, const Dev& d, int nsm, cudaStream_t s, int initial, int bpsm) {
  using S = ReconShape<M, GG>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_recon_coop<M, GG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::bytes);
    attr = true;
  }
  const int need = (d.ne + S::G - 1) / S::G;
  const int grid = initial ? need : std::min(need, nsm * bpsm);
  k_recon_coop<M, GG><<<grid, S::kThreads, S::bytes, s>>>(T, d, initial);
}

template <int M>
void launch_recon(const Tab& T, const Dev& d, int nsm, cudaStream_t s, int initial, const Tiles& tl) {
  constexpr int G0 = recon_g_default<M>();
  if (tl.recon_half) launch_recon_g<M, G0 / 2>(T, d, nsm, s, initial, tl.bpsm);
  else launch_recon_g<M, G0>(T, d, nsm, s, initial, tl.bpsm);
}

template <int M, int TH>
void launch_predict_t(const Tab& T, const Dev& d, int nsm, cudaStream_t s, int initial, int bpsm) {
  using S = PredShape<M, TH>;
  const int need = (d.ne + S::G - 1) / S::G;
  // sweeps: the blocks that fit on the GPU at once (the launch bounds' two or
  // three per SM), so that balanced rounds give every SM the same elements
  const int grid = initial ? need : std::min(need, nsm * (TH >= 256 ? 2 : 3));
  (void)bpsm;
  k_predict_coop<M, TH><<<grid, S::kThreads, 0, s>>>(T, d, initial, T.gts);
}

template <int M>
void launch_predict(const Tab& T, const Dev& d, int nsm, cudaStream_t s, int initial, const Tiles& tl) {
  if (tl.pred_wide) launch_predict_t<M, 256>(T, d, nsm, s, initial, tl.bpsm);
  else launch_predict_t<M, 128>(T, d, nsm, s, initial, tl.bpsm);
}

// ev (optional): kNumKernels + 1 events recorded on s around the launches,
// for per-kernel CUDA-event timing on the launching stream.
template <int M>
void sweep_impl(const Tab& T, const Dev& d, int nsm, cudaStream_t s, cudaEvent_t* ev, const Tiles& tl,
                cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  const int grid_all_e = (d.ne + kBlock - 1) / kBlock;
  const int grid_w = nsm * tl.bpsm;
  int k = 0;
  // external record nodes when captured into a graph (a plain record would only
  // order the capture)
  auto mark = [&]() { if (ev) cudaEventRecordWithFlags(ev[k++], s, cudaEventRecordExternal); };
  mark(); k_ready<<<std::min(grid_all_e * 8, nsm * 64), 256, 0, s>>>(T, d);
  if (!ev && side && fork && join) {
    // the node solver and the edge marking both read only the moved-node
    // list and write disjoint arrays: two branches of the graph
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    k_nodes_grp<M><<<grid_w * 2, kBlock, 0, side>>>(T, d);
    cudaEventRecord(join, side);
    k_edges<<<grid_w, kBlock, 0, s>>>(d);
    cudaStreamWaitEvent(s, join, 0);
  } else {
    mark(); k_nodes_grp<M><<<grid_w * 2, kBlock, 0, s>>>(T, d);
    mark(); k_edges<<<grid_w, kBlock, 0, s>>>(d);
  }
  mark(); k_flux_grp<M><<<grid_w * 4, kBlock, 0, s>>>(T, d);
  mark(); k_update<<<grid_w, kBlock, 0, s>>>(T, d);
  mark(); launch_recon<M>(T, d, nsm, s, 0, tl);
  mark(); launch_predict<M>(T, d, nsm, s, 0, tl);
  mark(); k_finish<<<grid_w, kBlock, 0, s>>>(T, d);
  mark();
}

template <int M>
void initial_impl(const Tab& T, const Dev& d, int nsm, cudaStream_t s, const Tiles& tl) {
  k_fill_counters_initial<<<1, 32, 0, s>>>(d);
  launch_recon<M>(T, d, nsm, s, 1, tl);
  launch_predict<M>(T, d, nsm, s, 1, tl);
}

template <int M>
void sync_cut_impl(const Tab& T, const Dev& d, int nsm, cudaStream_t s, long long Tn, const Tiles& tl) {
  k_sync_done<<<1, 32, 0, s>>>(d);
  k_sync_cut<M><<<nsm * 4, 256, 0, s>>>(d, Tn);
  launch_predict<M>(T, d, nsm, s, 0, tl);
  k_sync_done<<<1, 32, 0, s>>>(d);
}

template <int M>
void sync_resume_impl(const Tab& T, const Dev& d, int nsm, cudaStream_t s, long long Told, const Tiles& tl) {
  k_sync_done<<<1, 32, 0, s>>>(d);
  k_sync_resume<<<nsm * 4, 256, 0, s>>>(d, Told);
  launch_recon<M>(T, d, nsm, s, 0, tl);
  launch_predict<M>(T, d, nsm, s, 0, tl);
  k_sync_done<<<1, 32, 0, s>>>(d);
}

template <int M>
void lists_impl(const Tab& T, const Dev& d, int nsm, cudaStream_t s) {
  const int grid_all_e = (d.ne + kBlock - 1) / kBlock;
  const int grid_w = nsm * 8;
  k_ready<<<std::min(grid_all_e * 8, nsm * 64), 256, 0, s>>>(T, d);
  k_nodes_grp<M><<<grid_w * 2, kBlock, 0, s>>>(T, d);
  k_edges<<<grid_w, kBlock, 0, s>>>(d);
}

__global__ void k_dfma_chain(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

const char* kernel_name(int k) {
  static const char* names[kNumKernels] = {"k_ready", "k_nodes", "k_edges", "k_flux",
                                           "k_update", "k_recon", "k_predict", "k_finish"};
  return (k >= 0 && k < kNumKernels) ? names[k] : nullptr;
}

void launch_sweep(const Tab& T, const Dev& d, int nsm, cudaStream_t s, cudaEvent_t* ev, const Tiles& tl,
                  cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  switch (T.M) {
    case 1: sweep_impl<1>(T, d, nsm, s, ev, tl, side, fork, join); break;
    case 2: sweep_impl<2>(T, d, nsm, s, ev, tl, side, fork, join); break;
    default: sweep_impl<3>(T, d, nsm, s, ev, tl, side, fork, join); break;
  }
}

void launch_initial(const Tab& T, const Dev& d, int nsm, cudaStream_t s, const Tiles& tl) {
  switch (T.M) {
    case 1: initial_impl<1>(T, d, nsm, s, tl); break;
    case 2: initial_impl<2>(T, d, nsm, s, tl); break;
    default: initial_impl<3>(T, d, nsm, s, tl); break;
  }
}

void launch_phase_a_lists(const Tab& T, const Dev& d, int nsm, cudaStream_t s) {
  switch (T.M) {
    case 1: lists_impl<1>(T, d, nsm, s); break;
    case 2: lists_impl<2>(T, d, nsm, s); break;
    default: lists_impl<3>(T, d, nsm, s); break;
  }
}

void launch_sync_cut(const Tab& T, const Dev& d, int nsm, cudaStream_t s, long long Tn, const Tiles& tl) {
  switch (T.M) {
    case 1: sync_cut_impl<1>(T, d, nsm, s, Tn, tl); break;
    case 2: sync_cut_impl<2>(T, d, nsm, s, Tn, tl); break;
    default: sync_cut_impl<3>(T, d, nsm, s, Tn, tl); break;
  }
}

void launch_sync_resume(const Tab& T, const Dev& d, int nsm, cudaStream_t s, long long Told, const Tiles& tl) {
  switch (T.M) {
    case 1: sync_resume_impl<1>(T, d, nsm, s, Told, tl); break;
    case 2: sync_resume_impl<2>(T, d, nsm, s, Told, tl); break;
    default: sync_resume_impl<3>(T, d, nsm, s, Told, tl); break;
  }
}

void launch_products(const Tab& T, const Dev& d, int nsm, cudaStream_t s) {
  switch (T.M) {
    case 1: k_products<1><<<nsm * 4, 64, 0, s>>>(T, d); break;
    case 2: k_products<2><<<nsm * 4, 64, 0, s>>>(T, d); break;
    default: k_products<3><<<nsm * 4, 64, 0, s>>>(T, d); break;
  }
}

// Dependent DFMA chains (8 per thread) over 4 x 256 threads per SM.
double measure_fp64_peak() {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  const int blocks = nsm * 4, threads = 256, iters = 8192;
  double* out = nullptr;
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return -1;
  if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) { cudaStreamDestroy(s); return -1; }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    k_dfma_chain<<<blocks, threads, 0, s>>>(out, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaStreamDestroy(s);
  if (!ok) return -1;
  return 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e9;
}

}  // namespace aw
